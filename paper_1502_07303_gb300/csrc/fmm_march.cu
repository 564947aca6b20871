// fmm_march.cu -- forward kernels of the restarted narrow band fast marching
// method (Yang & Stern), brick decomposition on one GB300 (sm_103a).
//
// Mapping of the paper's parallel algorithm (Sec. 4) onto the GPU:
//   subdomain Omega_p + ghost layer Theta_p  -> one 8x8x8 brick staged with its
//                                               face halo in shared memory
//   Initialize_Interface_Parallel (Alg. 8)  -> k_init_sources / k_init_reinit
//   Initialize_Heap_Parallel (Alg. 9)       -> k_march<mode 0> (one relax of
//                                               every cell next to a FIX cell)
//   local minima + AllReduce (Alg. 16)      -> k_reduce + k_control
//   March_Narrow_Band_Parallel (Alg. 12)    -> march_brick, run by one of three
//                                               restart schedules (below)
//   Collect/Exchange/Integrate (Alg. 13-15) -> write-back to HBM plus per-face
//                                               "fresh" bit masks on the
//                                               neighbour brick, whose next
//                                               staging reads the new values
//   second march of Alg. 16                 -> the neighbour is marched again
//                                               (queued, or listed as dirty)
//
// Restart schedules: continuous (k_march_continuous: one launch for the whole
// solve, bricks from a device-side queue, the bound raised in the kernel when
// a restart runs out of parallel work), persistent (k_seed +
// k_march_persistent: one queue-driven launch per restart) and phased
// (k_select + k_march<mode 1>: one launch per pass over a work list).
//
// Inside a brick (one warp per brick) the heap of Algorithm 12 is replaced by
// a bucketed, label-correcting march: each round accepts every BAND cell whose |psi| is
// within a bucket width of the brick's BAND minimum (and within the restart
// bound), then every cell next to a newly accepted cell re-solves Algorithm
// 11.  A cell whose value drops is reset to BAND even if it was accepted,
// exactly as Algorithm 10 resets KNOWN_NEW/KNOWN_OLD points, so the march
// ends at the same local fixed point as the heap march.
//
// A brick never solves cells it does not own: halo cells are read-only
// upwind data.  Every cell therefore has a single writer, and values only
// decrease, so a halo read that races with the owner's write-back can only
// return an upper bound; the owner then flags the change and the brick is
// marched again before termination can be declared.
#include "fmm_internal.h"
#include "fmm_queue.cuh"
#include "fmm_fp64.cuh"
#include "fmm_df.cuh"
#include "fmm_lanes.cuh"

#include <cfloat>
#include <cmath>
#include <math_constants.h>
#include <type_traits>

namespace fmmgb {
namespace {

template <typename real>
__device__ __forceinline__ real inf_v();
template <>
__device__ __forceinline__ float inf_v<float>() { return __int_as_float(0x7f800000); }
template <>
__device__ __forceinline__ double inf_v<double>() { return __longlong_as_double(0x7ff0000000000000ll); }

__device__ __forceinline__ bool is_known(uint8_t tg) { return (tg & ST_MASK) >= ST_KNOWN; }

__device__ __forceinline__ void brick_coords(const Geom &g, long long b, int &bx, int &by,
                                             int &bz)
{
    bx = (int)(b % g.nbx);
    long long r = b / g.nbx;
    by = (int)(r % g.nby);
    bz = (int)(r / g.nby);
}

// Brick across face f (0..5 = -x, +x, -y, +y, -z, +z) of brick b, or -1.  A
// batch of grids stores a neighbour table (no neighbour across the border of
// a grid); a single grid computes it from the brick coordinates.
__device__ __forceinline__ long long neighbour_brick(const Geom &g, const int *nbr, long long b,
                                                    int f)
{
    if (nbr)
        return (long long)nbr[b * kFaces + f];
    int bx, by, bz;
    brick_coords(g, b, bx, by, bz);
    const int axis = f >> 1, dir = (f & 1) ? 1 : -1;
    const int nbx = bx + (axis == 0 ? dir : 0);
    const int nby = by + (axis == 1 ? dir : 0);
    const int nbz = bz + (axis == 2 ? dir : 0);
    if (nbx < 0 || nbx >= g.nbx || nby < 0 || nby >= g.nby || nbz < 0 || nbz >= g.nbz)
        return -1;
    return ((long long)nbz * g.nby + nby) * g.nbx + nbx;
}

// ---------------------------------------------------------------------------
// Algorithm 11 (Solve_Quadratic_Parallel) on a staged tile.
//
// kv holds the value of every KNOWN/FIX cell of the brick and its halo, +inf
// for an unknown halo cell and the marked (sign bit set) value of every other
// brick cell, so "G in KNOWN and |psi_n| < |psi_cell|" is "kv_n < Tc" on the
// unsigned bit patterns (klt).
// The per-axis choice and the nested upwind sets (each time dropping the
// largest psi_i) follow the algorithm.  Algorithm 11 keeps the smallest
// causal root over the sets; going from the full set down, the first causal
// root already is that minimum: a causal root t_S of a nested set S satisfies
// sum over all axes of max(t_S - psi_i, 0)^2 >= (h/F)^2, so t_S is never
// below the unique solution t* of sum max(t - psi_i, 0)^2 = (h/F)^2, and t*
// is the causal root of the set {i : psi_i < t*}.  The loop therefore stops
// at the first causal root.  set_out receives its upwind set (2 bits per
// axis: 1 = minus, 2 = plus neighbour).
//
// |psi| values are never negative, so double comparisons are done on the
// bit patterns (integer compares keep them off the FP64 pipe).
// ---------------------------------------------------------------------------

__device__ __forceinline__ bool lt(double a, double b)
{
    // valid for values >= 0 and +inf; a negative discriminant has the sign
    // bit set and compares below every non-negative value
    return __double_as_longlong(a) < __double_as_longlong(b);
}
__device__ __forceinline__ bool lt(float a, float b) { return a < b; }
__device__ __forceinline__ double vmin(double a, double b) { return lt(a, b) ? a : b; }
__device__ __forceinline__ float vmin(float a, float b) { return fminf(a, b); }

// Tile entries of the march: a known value as it is, any other brick cell
// with its sign bit set (the "not known" mark, see WarpTile).  Compared as
// unsigned bit patterns, a marked entry orders above every value including
// +inf, so the smaller of two neighbours is the known one and a marked
// entry is never below a cell's value: Algorithm 11's "known and smaller"
// test costs no decoding.
__device__ __forceinline__ bool klt(double a, double b)
{
    return (unsigned long long)__double_as_longlong(a) < (unsigned long long)__double_as_longlong(b);
}
__device__ __forceinline__ bool klt(float a, float b) { return __float_as_uint(a) < __float_as_uint(b); }
__device__ __forceinline__ double kmin(double a, double b) { return klt(a, b) ? a : b; }
__device__ __forceinline__ float kmin(float a, float b)
{
    return __uint_as_float(umin(__float_as_uint(a), __float_as_uint(b)));
}
// mark / unmark (set / clear the sign bit, on the high word of a double)
__device__ __forceinline__ double kmark(double v)
{
    return __hiloint2double(__double2hiint(v) | (int)0x80000000, __double2loint(v));
}
__device__ __forceinline__ float kmark(float v) { return __uint_as_float(__float_as_uint(v) | 0x80000000u); }
__device__ __forceinline__ double kval(double v)
{
    return __hiloint2double(__double2hiint(v) & 0x7fffffff, __double2loint(v));
}
__device__ __forceinline__ float kval(float v) { return __uint_as_float(__float_as_uint(v) & 0x7fffffffu); }

// Double square root without the FP64 pipe's slow conversions (fmm_fp64.cuh).
__device__ __forceinline__ double vsqrt(double v) { return sqrt_fp64(v); }
// Single precision: x * rsqrt(x) (a few ulp, far below the fp32 tolerance;
// 0 stays 0).  The +inf speed term of an obstacle cell gives NaN, which fails
// every causality test of Algorithm 11, so the cell's candidate is +inf.
__device__ __forceinline__ float vsqrt(float v) { return v * rsqrtf(fmaxf(v, 1e-37f)); }

// The quadratic of Algorithm 11, sum_i (t - psi_i)^2 / h^2 = 1/F^2 over the
// upwind set, is solved for the unknown shifted by the smallest upwind value
// m: t = m + u, delta_i = psi_i - m, sum_i (u - delta_i)^2 = q with
// q = (h/F)^2.  The coefficients stay of order h, so rounding does not grow
// with psi (in psi itself b^2 and 4ac would cancel to ~3 (psi F/h)^2 ulp).
// The causality test psi_i < t is delta_i < u; the kernels that record the
// upwind sets for the adjoint make it on t = m + u and the values the cells
// hold (on rounded shifts delta_i < u can hold while t rounds to psi_i, and a
// recorded set must point strictly downhill).  q is the cell's speed term.
//
// Per axis the upwind value is the smaller known neighbour if it is below
// Tc; with a tape (kTape) the side it came from is kept as well (the minus
// side on a tie; without a tape the compiler drops the sides).  The per-axis values are sorted once (a stable sort, so
// equal values keep the lower axis first and the higher axis is dropped
// first).  The smallest has delta = 0, so only the other two enter
// S = sum delta_i and Q = sum delta_i^2 (a dropped axis contributes 0):
// disc = S^2 - k (Q - q), u = (S + sqrt(disc)) / k, causal when the largest
// remaining delta is below u (with a tape: when t = m + u exceeds the largest
// remaining value).  All lanes of a warp evaluate their full set
// together; a lane whose full set is not causal (about 1% of solves) goes
// round the loop again.
template <typename real>
__device__ __forceinline__ void cswap(real &a, unsigned &ca, real &b, unsigned &cb)
{
    if (lt(b, a)) {
        const real t = a;
        a = b;
        b = t;
        const unsigned c = ca;
        ca = cb;
        cb = c;
    }
}

template <typename real, bool kTape>
__device__ __forceinline__ real solve_cell(const real *kv, int ti, real Tc, real q,
                                           uint8_t &set_out)
{
    const int off[3] = {1, kTile, kTile * kTile};
    const real INF = inf_v<real>();
    real v[3];
    unsigned code[3];
    int nd = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const real vm = kv[ti - off[a]], vp = kv[ti + off[a]];
        const real w = kmin(vm, vp);
        const bool up = klt(w, Tc);
        v[a] = up ? w : INF;
        code[a] = up ? (klt(vp, vm) ? 2u : 1u) << (2 * a) : 0u;   // dead without a tape
        nd += up;
    }
    set_out = 0;
    if (nd == 0)
        return INF;
    if constexpr (!kTape && sizeof(real) == 4) {
        // without sides to carry along: a min / max network
        const float a = fminf(v[0], v[1]), b = fmaxf(v[0], v[1]);
        const float d = fminf(b, v[2]);
        v[2] = fmaxf(b, v[2]);
        v[0] = fminf(a, d);
        v[1] = fmaxf(a, d);
    } else {
        // stable sort of three (adjacent compare-exchange, strict less-than)
        cswap(v[0], code[0], v[1], code[1]);
        cswap(v[1], code[1], v[2], code[2]);
        cswap(v[0], code[0], v[1], code[1]);
    }
    const real m = v[0];
    if constexpr (sizeof(real) == 8) {
        // double grids: the root in double-float arithmetic (fmm_df.cuh),
        // unless the speed term is outside its range (an obstacle's +inf)
        if (in_float_range(q)) {
            double t = 0.0;
            const int k = df_shifted_root<kTape>(v[0], v[1], v[2], nd, q, t);
            if (k == 0)
                return INF;
            set_out = (uint8_t)(code[0] | (k >= 2 ? code[1] : 0u) | (k == 3 ? code[2] : 0u));
            return t;
        }
    }
    real d1 = nd >= 2 ? v[1] - m : (real)0;
    real d2 = nd >= 3 ? v[2] - m : (real)0;
#pragma unroll 1
    for (; nd != 0; --nd) {
        const real S = d1 + d2;
        const real Q = fma(d2, d2, d1 * d1);
        const real k = nd == 3 ? (real)3 : (nd == 2 ? (real)2 : (real)1);
        const real disc = fma(-k, Q - q, S * S);
        if (!lt(disc, (real)0)) {
            const real inv_k = nd == 3 ? (real)(1.0 / 3.0) : (nd == 2 ? (real)0.5 : (real)1);
            const real u = (S + vsqrt(disc)) * inv_k;
            // causal: the largest remaining delta is below u; with a tape,
            // the root above the largest value as the cells hold it (the
            // upwind sets recorded for the adjoint must point strictly
            // downhill); one value: u > 0
            const real t = m + u;
            const bool causal = kTape ? (nd == 1 ? lt((real)0, u) : lt(nd == 3 ? v[2] : v[1], t))
                                      : lt(nd == 3 ? d2 : d1, u);
            if (causal) {
                set_out = (uint8_t)(code[0] | (nd >= 2 ? code[1] : 0u) | (nd == 3 ? code[2] : 0u));
                return t;
            }
        }
        // drop the largest remaining value
        if (nd == 3)
            d2 = (real)0;
        else
            d1 = (real)0;
    }
    return INF;
}

// Algorithm 11 with cells of size h * hy * hz: h_i^2 (t - psi_i)^2 summed
// over the set equals F^-2, i.e. sum_i w_i (u - delta_i)^2 = q with
// w_i = (h / h_i)^2 (w_x = 1), q = (h/F)^2 and the same shift t = m + u.
// The per-axis values are sorted together with their weights (and sides);
// with K = sum w_i, S = sum w_i delta_i and Q = sum w_i delta_i^2 over the
// set, disc = S^2 - K (Q - q), evaluated as K q - sum_{i<j} w_i w_j
// (delta_i - delta_j)^2, and u = (S + sqrt(disc)) / K; the largest remaining
// value is dropped while the set is not causal, as above.
template <typename real>
__device__ __forceinline__ void cswap_w(real &a, real &wa, unsigned &ca, real &b, real &wb, unsigned &cb)
{
    if (lt(b, a)) {
        const real t = a, tw = wa;
        a = b;
        b = t;
        wa = wb;
        wb = tw;
        const unsigned c = ca;
        ca = cb;
        cb = c;
    }
}
__device__ __forceinline__ float vdiv(float a, float b) { return a / b; }
__device__ __forceinline__ double vdiv(double a, double b) { return div_fp64(a, b); }

template <typename real, bool kTape>
__device__ __forceinline__ real solve_cell_w(const real *kv, int ti, real Tc, real q, real wy,
                                             real wz, uint8_t &set_out)
{
    const int off[3] = {1, kTile, kTile * kTile};
    const real wax[3] = {(real)1, wy, wz};
    const real INF = inf_v<real>();
    real v[3], w[3];
    unsigned code[3];
    int nd = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const real vm = kv[ti - off[a]], vp = kv[ti + off[a]];
        const real mn = kmin(vm, vp);
        const bool up = klt(mn, Tc);
        v[a] = up ? mn : INF;
        w[a] = up ? wax[a] : (real)0;
        code[a] = up ? (klt(vp, vm) ? 2u : 1u) << (2 * a) : 0u;   // dead without a tape
        nd += up;
    }
    set_out = 0;
    if (nd == 0)
        return INF;
    // stable sort of three, each weight and side with its value
    cswap_w(v[0], w[0], code[0], v[1], w[1], code[1]);
    cswap_w(v[1], w[1], code[1], v[2], w[2], code[2]);
    cswap_w(v[0], w[0], code[0], v[1], w[1], code[1]);
    const real m = v[0];
    real d1 = nd >= 2 ? v[1] - m : (real)0;
    real d2 = nd >= 3 ? v[2] - m : (real)0;
    const real w0 = w[0];
    real w1 = nd >= 2 ? w[1] : (real)0;
    real w2 = nd >= 3 ? w[2] : (real)0;
#pragma unroll 1
    for (; nd != 0; --nd) {
        const real K = w0 + w1 + w2;
        const real S = fma(w1, d1, w2 * d2);
        // S^2 - K (Q - q) = K q - sum_{i<j} w_i w_j (delta_i - delta_j)^2
        // (Lagrange's identity): with unequal weights S^2 and K Q nearly
        // cancel, the pairwise form does not
        const real e = d1 - d2;
        const real P = fma(w0 * w1, d1 * d1, fma(w0 * w2, d2 * d2, (w1 * w2) * (e * e)));
        const real disc = fma(K, q, -P);
        if (!lt(disc, (real)0)) {
            const real u = vdiv(S + vsqrt(disc), K);
            const real t = m + u;   // causal as in solve_cell
            const bool causal = kTape ? (nd == 1 ? lt((real)0, u) : lt(nd == 3 ? v[2] : v[1], t))
                                      : lt(nd == 3 ? d2 : d1, u);
            if (causal) {
                set_out = (uint8_t)(code[0] | (nd >= 2 ? code[1] : 0u) | (nd == 3 ? code[2] : 0u));
                return t;
            }
        }
        // drop the largest remaining value with its weight
        if (nd == 3) {
            d2 = (real)0;
            w2 = (real)0;
        } else {
            d1 = (real)0;
            w1 = (real)0;
        }
    }
    return INF;
}

// Warp minimum of non-negative values (or +inf): their bit patterns order
// like the values, so the integer reductions of the warp do it exactly (a
// double in two steps, high word then low word).
__device__ __forceinline__ float warp_min(float v)
{
    return __uint_as_float(__reduce_min_sync(0xffffffffu, __float_as_uint(v)));
}
__device__ __forceinline__ double warp_min(double v)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const unsigned hi = __reduce_min_sync(0xffffffffu, (unsigned)(b >> 32));
    const unsigned lo =
        __reduce_min_sync(0xffffffffu, (unsigned)(b >> 32) == hi ? (unsigned)b : 0xffffffffu);
    return __longlong_as_double((long long)(((unsigned long long)hi << 32) | lo));
}

// ---------------------------------------------------------------------------
// Algorithm 8: interface initialisation, written directly in brick layout.
// ---------------------------------------------------------------------------

// The per-cell kernels below run one CTA of kInitThreads threads per brick
// (grid-stride over bricks), so the brick coordinates are computed once per
// brick, with 32-bit arithmetic (a grid has fewer than 2^31 bricks).
constexpr int kInitThreads = 256;

__device__ __forceinline__ void brick_xyz32(const Geom &g, int b, int &bx, int &by, int &bz)
{
    bx = b % g.nbx;
    const int r = b / g.nbx;
    by = r % g.nby;
    bz = r / g.nby;
}

template <typename real>
__global__ void __launch_bounds__(kInitThreads) k_init_sources(Geom g, real *T, uint8_t *tag)
{
    for (int b = blockIdx.x; b < (int)g.nbricks; b += gridDim.x) {
        int bx, by, bz;
        brick_xyz32(g, b, bx, by, bz);
        const long long base = (long long)b * kB3;
        for (int c = threadIdx.x; c < kB3; c += kInitThreads) {
            const int i = bx * kB + (c & 7), j = by * kB + ((c >> 3) & 7), k = bz * kB + (c >> 6);
            const bool out = i >= g.nx || j >= g.ny || k >= g.nz;
            T[base + c] = inf_v<real>();
            tag[base + c] = out ? (uint8_t)(TG_OUT | ST_FAR) : (uint8_t)ST_FAR;
        }
    }
}

template <typename real>
__global__ void k_set_sources(Geom g, const long long *src, long long n_src, real *T,
                              uint8_t *tag)
{
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n_src;
         s += (long long)gridDim.x * blockDim.x) {
        const int i = (int)src[3 * s], j = (int)src[3 * s + 1], k = (int)src[3 * s + 2];
        const long long b = ((long long)(k >> 3) * g.nby + (j >> 3)) * g.nbx + (i >> 3);
        const long long e = b * kB3 + (i & 7) + 8 * (j & 7) + 64 * (k & 7);
        T[e] = (real)0;
        tag[e] = ST_FIX;
    }
}

// Front cells of a level set: a 6-neighbour of the opposite sign marks the
// cell as adjacent to the interface; its value is sign * (sum_a d_a^-2)^-1/2
// with d_a the smaller linear-interpolation crossing distance on axis a.
__device__ __forceinline__ double rcp_sq(double d) { return __ddiv_rn(1.0, __dmul_rn(d, d)); }
__device__ __forceinline__ float rcp_sq(float d) { return 1.f / (d * d); }
__device__ __forceinline__ double inv_sqrt_exact(double v) { return __ddiv_rn(1.0, __dsqrt_rn(v)); }
__device__ __forceinline__ float inv_sqrt_exact(float v) { return 1.f / sqrtf(v); }
__device__ __forceinline__ double crossing(double fc, double fq, double h)
{
    return __dmul_rn(__ddiv_rn(fc, __dsub_rn(fc, fq)), h);
}
__device__ __forceinline__ float crossing(float fc, float fq, double h)
{
    return (fc / (fc - fq)) * (float)h;
}

__device__ __forceinline__ bool nonneg(double v)
{
    // sign bit clear, or -0, tested on the high word (and the low word for -0)
    const int hi = __double2hiint(v);
    return hi >= 0 || (hi == (int)0x80000000 && __double2loint(v) == 0);
}
__device__ __forceinline__ bool nonneg(float v)
{
    const unsigned b = __float_as_uint(v);
    return (b >> 31) == 0u || (b << 1) == 0u;
}

// Algorithm 8 for one cell (i, j, k) of an nx*ny*nz level set with cells of
// size hx * hy * hz (the crossing distance of an axis is a fraction of that
// axis's cell size).  The level set may extend zlo layers below z = 0 and zhi
// layers above z = nz - 1 (phi points at layer 0): a subdomain of a
// decomposed grid sees the layers beyond its ghost layers, so its interface
// cells are those of the whole grid.  reinit_load reads the cell and its six
// neighbours (a neighbour outside the grid reads the cell itself, which never
// changes sign), reinit_eval computes psi and the tag from them; a kernel
// issues the loads of all its cells before the first evaluation.
template <typename real>
__device__ __forceinline__ void reinit_load(const real *__restrict__ phi, int nx, int ny, int nz, int i,
                                            int j, int k, int zlo, int zhi, real &fc, real fn[6])
{
    const long long sx = 1, sy = nx, sz = (long long)nx * ny;
    const long long p = (long long)k * sz + (long long)j * sy + i;
    fc = phi[p];
    const int co[3] = {i, j, k};
    const int lo[3] = {0, 0, -zlo};
    const int ext[3] = {nx, ny, nz + zhi};
    const long long st[3] = {sx, sy, sz};
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const int dir = s ? 1 : -1;
            const int q = co[a] + dir;
            const long long off = (q < lo[a] || q >= ext[a]) ? 0ll : (dir < 0 ? -st[a] : st[a]);
            fn[2 * a + s] = phi[p + off];
        }
}

template <typename real>
__device__ __forceinline__ void reinit_eval(real fc, const real fn[6], double hx, double hy, double hz,
                                            real &Tv, uint8_t &tg)
{
    const double hs[3] = {hx, hy, hz};
    // sign tests on the bit patterns (phi >= 0: sign bit clear, or -0): the
    // FP64 pipe's comparisons would bound the whole pass for double grids
    const bool pos = nonneg(fc);
    real d[3];
    bool any = false;
    bool cross[6];
#pragma unroll
    for (int n = 0; n < 6; ++n) {
        cross[n] = nonneg(fn[n]) != pos;
        any = any || cross[n];
    }
    if (!any) {
        Tv = inf_v<real>();
        tg = pos ? (uint8_t)ST_FAR : (uint8_t)(ST_FAR | TG_NEG);
        return;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        d[a] = inf_v<real>();
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            if (!cross[2 * a + s])
                continue;
            const real dist = crossing(fc, fn[2 * a + s], hs[a]);
            if (dist < d[a])
                d[a] = dist;
        }
    }
    real inv = (real)0;
    bool zero = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (d[a] == inf_v<real>())
            continue;
        if (d[a] == (real)0)
            zero = true;
        else
            inv = inv + rcp_sq(d[a]);
    }
    Tv = zero ? (real)0 : inv_sqrt_exact(inv);
    tg = pos ? (uint8_t)ST_FIX : (uint8_t)(ST_FIX | TG_NEG);
}

template <typename real>
__device__ __forceinline__ void reinit_cell(const real *__restrict__ phi, int nx, int ny, int nz,
                                            int i, int j, int k, double hx, double hy, double hz,
                                            real &Tv, uint8_t &tg, int zlo = 0, int zhi = 0)
{
    real fc, fn[6];
    reinit_load<real>(phi, nx, ny, nz, i, j, k, zlo, zhi, fc, fn);
    reinit_eval<real>(fc, fn, hx, hy, hz, Tv, tg);
}

template <typename real>
__global__ void __launch_bounds__(kInitThreads) k_init_reinit(Geom g, double hx, double hy, double hz,
                                                              const real *__restrict__ phi, real *T,
                                                              uint8_t *tag, int zlo, int zhi)
{
    static_assert(kB3 == 2 * kInitThreads, "two cells per thread");
    for (int b = blockIdx.x; b < (int)g.nbricks; b += gridDim.x) {
        int bx, by, bz;
        brick_xyz32(g, b, bx, by, bz);
        const long long base = (long long)b * kB3;
        // cells c and c + 256 of the brick: z and z + 4
        const int c = threadIdx.x;
        const int i = bx * kB + (c & 7), j = by * kB + ((c >> 3) & 7), k = bz * kB + (c >> 6);
        const bool in0 = i < g.nx && j < g.ny && k < g.nz;
        const bool in1 = i < g.nx && j < g.ny && k + 4 < g.nz;
        real fc0 = (real)0, fc1 = (real)0, fn0[6], fn1[6];
        if (in0)
            reinit_load<real>(phi, g.nx, g.ny, g.nz, i, j, k, zlo, zhi, fc0, fn0);
        if (in1)
            reinit_load<real>(phi, g.nx, g.ny, g.nz, i, j, k + 4, zlo, zhi, fc1, fn1);
        real Tv0 = inf_v<real>(), Tv1 = inf_v<real>();
        uint8_t tg0 = TG_OUT | ST_FAR, tg1 = TG_OUT | ST_FAR;
        if (in0)
            reinit_eval<real>(fc0, fn0, hx, hy, hz, Tv0, tg0);
        if (in1)
            reinit_eval<real>(fc1, fn1, hx, hy, hz, Tv1, tg1);
        T[base + c] = Tv0;
        tag[base + c] = tg0;
        T[base + c + kInitThreads] = Tv1;
        tag[base + c + kInitThreads] = tg1;
    }
}

// Speed field to brick layout: the speed term (h/F)^2 of the shifted solve
// (h the x cell size).  Each brick also records its bucket width
// hmin * min(1/F) / sqrt(3), hmin the smallest cell size.
__device__ __forceinline__ double speed_term(double F, double h) { return (h * h) / (F * F); }
__device__ __forceinline__ float speed_term(float F, double h)
{
    const float hf = (float)h;
    return (hf * hf) / (F * F);
}

template <typename real>
__global__ void __launch_bounds__(kThreads) k_load_speed(Geom g, double h, double hmin,
                                                         const real *__restrict__ speed,
                                                         double speed_const, real *spd, real *bdelta,
                                                         Control *ctrl)
{
    __shared__ real red[kThreads / 32];
    const int t = threadIdx.x;
    for (long long b = blockIdx.x; b < g.nbricks; b += gridDim.x) {
        int bx, by, bz;
        brick_coords(g, b, bx, by, bz);
        const int i = bx * kB + (t & 7), j = by * kB + ((t >> 3) & 7), k = bz * kB + (t >> 6);
        const bool out = i >= g.nx || j >= g.ny || k >= g.nz;
        real F = (real)speed_const;
        if (speed && !out)
            F = speed[((long long)k * g.ny + j) * g.nx + i];
        if (out)
            F = (real)1;
        // F = 0: an obstacle cell, whose speed term (h/F)^2 is +inf, so no
        // solve ever gives it a finite value
        if (!(F >= (real)0) || !(F < inf_v<real>()))
            atomicOr(&ctrl->error, ERR_SPEED);
        if (spd)
            spd[b * kB3 + t] = speed_term(F, h);
        real fm = out ? (real)0 : F;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            fm = fmax(fm, __shfl_xor_sync(0xffffffffu, fm, o));
        if ((t & 31) == 0)
            red[t >> 5] = fm;
        __syncthreads();
        if (t == 0) {
            real m = red[0];
            for (int w = 1; w < kThreads / 32; ++w)
                m = fmax(m, red[w]);
            if (!(m > (real)0))
                m = (real)speed_const;
            bdelta[b] = (real)(hmin / (1.7320508075688772 * (double)m));
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// The brick march: one warp per brick.  kMode 0: Algorithm 9 over all bricks
// (every non-FIX cell next to a known cell is solved once, nothing is
// accepted).  kMode 1: Algorithm 12 up to the restart bound over the bricks
// of work list `which`.
//
// Lane l owns the 16 cells c = l + 32 k (k = 0..15) of the brick: x = l % 8,
// y = (l / 8) % 4 + 4 (k % 2), z = k / 2.  Cell sets (BAND, KNOWN, frozen,
// side, accepted, to-solve) are 16-bit masks per lane, bit k for cell
// l + 32 k, so the per-round passes touch only the cells in a set.  The cells
// to solve in a round are compacted into a list by a warp prefix sum, so all
// 32 lanes solve.
// ---------------------------------------------------------------------------

#ifndef FMM_MARCH_BLOCKS_F32
#define FMM_MARCH_BLOCKS_F32 7
#endif
#ifndef FMM_MARCH_BLOCKS_F64
#define FMM_MARCH_BLOCKS_F64 5
#endif
#ifndef FMM_MARCH_BLOCKS_F64_TAPE
#define FMM_MARCH_BLOCKS_F64_TAPE 5
#endif
// Resident CTAs per SM the march kernels are compiled for (registers); the
// warp tiles (5.1 / 5.6 KB in float, 9.0 / 9.5 KB in double, without / with
// the tape) allow these as well.  Measured on the 1024^3 sphere: fp64 with
// 4 / 5 / 6 CTAs 261 / 236 / 242 ms (six leave 80 registers and spill),
// fp32 with 6 / 7 / 8 CTAs 122 / 115 / 115 ms (eight slow the 256^3 case).
template <typename real, bool kTape>
constexpr int march_min_blocks()
{
    return sizeof(real) == 4 ? FMM_MARCH_BLOCKS_F32 : (kTape ? FMM_MARCH_BLOCKS_F64_TAPE : FMM_MARCH_BLOCKS_F64);
}
constexpr unsigned FULL = 0xffffffffu;

// The brick and its face halo in one 10^3 tile (x fastest), shifted by one
// entry so that every row of 8 brick cells starts on a 16-byte boundary in
// double and an 8-byte boundary in float: kMT0 is the tile index of brick
// cell (0, 0, 0), kMH0 that of halo position (0, 0, 0).  A brick cell holds
// its current |psi|, with the sign bit set unless the cell is KNOWN or FIX; a
// halo cell holds the neighbour's known value or +inf.  One array for the
// known values and the current values keeps the fp64 tile at 9.5 KB a warp,
// which lets five CTAs of four warps share an SM.
constexpr int kMH0 = 1;
constexpr int kMT0 = kMH0 + 1 + kTile + kTile * kTile;
constexpr int kMTile = kMH0 + kTile3 + 1;

__device__ __forceinline__ int mt_of(int c)
{
    return kMT0 + (c & 7) + kTile * ((c >> 3) & 7) + kTile * kTile * (c >> 6);
}

template <typename real, bool kTape>
struct WarpTile {
    alignas(16) real kv[kMTile];       // brick (marked unless known) and face halo
    alignas(16) uint8_t tp[kTape ? kB3 : 16];   // upwind sets (with a tape)
    alignas(16) uint16_t list[kB3];    // compacted cells to solve (the tags
                                       // while staging and writing back)
    unsigned improved[32]; // per owner lane: cells whose value dropped
};
static_assert(sizeof(WarpTile<float, false>) % 16 == 0 && sizeof(WarpTile<double, false>) % 16 == 0 &&
                  sizeof(WarpTile<float, true>) % 16 == 0 && sizeof(WarpTile<double, true>) % 16 == 0,
              "every warp's tile starts on a 16-byte boundary");
static_assert((kMT0 * 8) % 16 == 0 && (kTile * 8) % 16 == 0 && (kMT0 * 4) % 8 == 0 && (kTile * 4) % 8 == 0,
              "brick rows of the tile start on 16 (double) / 8 (float) byte boundaries");

// The q-th 16 bytes of a brick in brick order (cells c = x + 8 y + 64 z) to
// and from the tile rows: two cells per 16 bytes in double (four per row),
// four in float (two per row, stored as two 8-byte halves).  row_load clears
// the marks: the brick in global memory holds |psi|.
__device__ __forceinline__ void row_store(double *kv, int q, uint4 x)
{
    const int row = q >> 2;   // y + 8 z
    reinterpret_cast<uint4 *>(kv + kMT0 + kTile * (row & 7) + kTile * kTile * (row >> 3))[q & 3] = x;
}
__device__ __forceinline__ void row_store(float *kv, int q, uint4 x)
{
    const int row = q >> 1;
    uint2 *d = reinterpret_cast<uint2 *>(kv + kMT0 + kTile * (row & 7) + kTile * kTile * (row >> 3) + 4 * (q & 1));
    d[0] = make_uint2(x.x, x.y);
    d[1] = make_uint2(x.z, x.w);
}
__device__ __forceinline__ uint4 row_load(const double *kv, int q)
{
    const int row = q >> 2;
    uint4 x = reinterpret_cast<const uint4 *>(kv + kMT0 + kTile * (row & 7) + kTile * kTile * (row >> 3))[q & 3];
    x.y &= 0x7fffffffu;   // high words
    x.w &= 0x7fffffffu;
    return x;
}
__device__ __forceinline__ uint4 row_load(const float *kv, int q)
{
    const int row = q >> 1;
    const uint2 *d =
        reinterpret_cast<const uint2 *>(kv + kMT0 + kTile * (row & 7) + kTile * kTile * (row >> 3) + 4 * (q & 1));
    const uint2 a = d[0], b = d[1];
    return make_uint4(a.x & 0x7fffffffu, a.y & 0x7fffffffu, b.x & 0x7fffffffu, b.y & 0x7fffffffu);
}

// Cells of lane l next to a halo cell flagged in the per-face masks F[6]
// (face bit = u + 8 v with (u, v) the two in-face coordinates).
__device__ __forceinline__ unsigned face_mask(const unsigned long long F[kFaces], int lane)
{
    const int x = lane & 7, r = (lane >> 3) & 3;
    unsigned n = 0;
#pragma unroll 4
    for (int k = 0; k < 16; ++k) {
        const int y = r + 4 * (k & 1), z = k >> 1;
        bool hit = false;
        if (x == 0)
            hit = hit || ((F[0] >> (y + 8 * z)) & 1ull);
        if (x == 7)
            hit = hit || ((F[1] >> (y + 8 * z)) & 1ull);
        if (y == 0)
            hit = hit || ((F[2] >> (x + 8 * z)) & 1ull);
        if (y == 7)
            hit = hit || ((F[3] >> (x + 8 * z)) & 1ull);
        if (z == 0)
            hit = hit || ((F[4] >> (x + 8 * y)) & 1ull);
        if (z == 7)
            hit = hit || ((F[5] >> (x + 8 * y)) & 1ull);
        if (hit)
            n |= 1u << k;
    }
    return n;
}

struct MarchStats {
    unsigned long long marches, rounds, accepted, exchanges, solves;
};

// One brick march.  F_in: the halo cells whose known value changed since the
// brick last ran (kMode 1); kMode 0 derives them from the known halo cells.
// kFresh: read the brick and halo through L2 (the persistent kernel, where the
// brick may have been written by another SM during the same launch).  kTape:
// record the upwind set of every solve for the adjoint (without it the
// compiler drops the set bookkeeping of Algorithm 11 altogether).  kAniso:
// cells of unequal sizes (the weighted solve).  On
// return, lanes 0..5 hold in notify_m / notify_nb the changed boundary cells
// and the neighbour brick across face = lane (mode 1), and every lane holds in
// notify_v[2] the smallest flagged value of each side (+inf: none).
template <typename real, bool kHetero, int kMode, bool kFresh, bool kTape, bool kAniso>
__device__ __forceinline__ void march_brick(const Geom &g, const DeviceState &s, const SolveParams &p,
                                            double spd_const_term, WarpTile<real, kTape> &W, long long b,
                                            const unsigned long long *F_in, real bound0, real bound1,
                                            int lane, unsigned long long &notify_m,
                                            long long &notify_nb, real *notify_v, MarchStats &st)
{
    real *T = (real *)s.T;
    uint8_t *tag = s.tag;
    const real *spd = (const real *)s.spd;
    const real *bdelta = (const real *)s.bdelta;
    real *bmin = (real *)s.bmin;
    const real INF = inf_v<real>();
    const int lx = lane & 7, lr = (lane >> 3) & 3;
    const int tb = kMT0 + lx + kTile * lr;   // tile index of the lane's cell k = 0
    long long nbi[kFaces];
#pragma unroll
    for (int f = 0; f < kFaces; ++f)
        nbi[f] = neighbour_brick(g, s.nbr, b, f);
    const long long base = b * kB3;

    // ---- stage the brick ---------------------------------------------------
    // The brick's values, tags (and tape) are contiguous: 16-byte loads copy
    // them into shared memory (the values into the rows of the tile, the tags
    // into the list buffer, unused until the rounds), then every lane marks
    // its own cells there.
    uint8_t *const stag = reinterpret_cast<uint8_t *>(W.list);
    {
        constexpr int kVecs = kB3 * (int)sizeof(real) / 16 / 32;   // 16-byte loads per lane
        const uint4 *gv = reinterpret_cast<const uint4 *>(T + base);
#pragma unroll
        for (int j = 0; j < kVecs; ++j) {
            const int q = lane + 32 * j;
            const uint4 x = kFresh ? __ldcg(gv + q) : gv[q];
            row_store(W.kv, q, x);
        }
        const uint4 *gt = reinterpret_cast<const uint4 *>(tag + base);
        reinterpret_cast<uint4 *>(stag)[lane] = kFresh ? __ldcg(gt + lane) : gt[lane];
        if (kTape) {
            const uint4 *gp = reinterpret_cast<const uint4 *>(s.tape + base);
            reinterpret_cast<uint4 *>(W.tp)[lane] = kFresh ? __ldcg(gp + lane) : gp[lane];
        }
    }
    __syncwarp();
    unsigned band = 0, known = 0, fix = 0, out = 0, neg = 0;
    real r0 = INF, r1 = INF;   // lane minimum of the BAND cells of each side
#pragma unroll 4
    for (int k = 0; k < 16; ++k) {
        const int c = lane + 32 * k;
        const int ti = tb + 40 * (k & 1) + 100 * (k >> 1);
        const real v = W.kv[ti];
        const uint8_t t = stag[c];
        const uint8_t sv = t & ST_MASK;
        if (sv < ST_KNOWN)
            W.kv[ti] = kmark(v);
        band |= (unsigned)(sv == ST_BAND) << k;
        known |= (unsigned)(sv >= ST_KNOWN) << k;
        fix |= (unsigned)(sv == ST_FIX) << k;
        out |= (unsigned)((t & TG_OUT) != 0) << k;
        neg |= (unsigned)((t & TG_NEG) != 0) << k;
        if (sv == ST_BAND) {
            if (t & TG_NEG)
                r0 = vmin(r0, v);
            else
                r1 = vmin(r1, v);
        }
    }
    W.improved[lane] = 0u;
    const unsigned frozen = fix | out;
    // ---- halo: the face layers of the six neighbours (read-only) ----------
    unsigned long long F[kFaces];
#pragma unroll
    for (int f = 0; f < kFaces; ++f)
        F[f] = kMode == 0 ? 0ull : F_in[f];
#pragma unroll
    for (int f = 0; f < kFaces; ++f) {
        const long long nb = nbi[f];
        const int axis = f >> 1, dir = (f & 1) ? 1 : -1;
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const int q = lane + 32 * half, u = q & 7, v = q >> 3;
            real val = INF;
            if (kMode == 1 && nb >= 0 && s.faces) {
                // deterministic mode: the neighbour's layer as of the last pass
                val = __ldcg((const real *)s.faces + nb * (kFaces * 64) + (f ^ 1) * 64 + q);
            } else if (nb >= 0) {
                const int edge = dir < 0 ? kB - 1 : 0;
                const int cx = axis == 0 ? edge : u;
                const int cy = axis == 1 ? edge : (axis == 0 ? u : v);
                const int cz = axis == 2 ? edge : v;
                const long long ci = nb * kB3 + cx + kB * cy + kB * kB * cz;
                const uint8_t ntg = __ldcg(tag + ci);
                const real nv = __ldcg(T + ci);
                if (is_known(ntg))
                    val = nv;
            }
            const int hedge = dir < 0 ? 0 : kTile - 1;
            const int hx = axis == 0 ? hedge : u + 1;
            const int hy = axis == 1 ? hedge : (axis == 0 ? u + 1 : v + 1);
            const int hz = axis == 2 ? hedge : v + 1;
            W.kv[kMH0 + hx + kTile * hy + kTile * kTile * hz] = val;
            if (kMode == 0) {
                // Algorithm 9: every known halo cell updates its neighbours
                const unsigned bal = __ballot_sync(FULL, lt(val, INF));
                F[f] |= (unsigned long long)bal << (32 * half);
            }
        }
    }
    __syncwarp();

    unsigned relax = face_mask(F, lane);
    if (kMode == 0)
        relax |= neighbour_mask(known, lane);
    relax &= ~frozen;

    const real delta = (real)p.bucket * bdelta[b];
    unsigned acc_any = 0;
    int rounds = 0;
    real m0 = INF, m1 = INF;
    // Settled cells: KNOWN cells at or below the band minimum of their side.
    // An accepted value is at least the band minimum of its round, and an
    // update from an upwind value v never goes below v, so while the minimum
    // does not fall no later acceptance can lower a settled cell and the
    // cell is left out of the solves.  The minimum normally only rises (a
    // value computed from an accepted neighbour v is a causal root above v),
    // but a halo value staged before its change flag arrived (written by a
    // neighbour brick during this march) can let a relaxed cell drop below it;
    // when the minimum of a side falls, that side's settled cells are
    // released.  pend: cells accepted at or below the largest lim so far
    // (pl0, pl1) that settle once the minimum of their side reaches it.
    unsigned settled = 0, pend = 0;
    real pl0 = (real)0, pl1 = (real)0;
    real mp0 = (real)0, mp1 = (real)0;   // band minima of the previous round
    for (;;) {
        // compact the cells to solve (warp prefix sum of the lane counts)
        const int cnt = __popc(relax);
        int pre = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(FULL, pre, o);
            if (lane >= o)
                pre += t;
        }
        const int n_items = __shfl_sync(FULL, pre, 31);
        pre -= cnt;
        st.solves += (unsigned long long)n_items;
        for (unsigned m = relax; m; m &= m - 1u)
            W.list[pre++] = (uint16_t)(lane + 32 * (__ffs(m) - 1));
        __syncwarp();
        // Algorithm 10/11: solve, then apply (Jacobi within 32 cells)
        for (int i0 = 0; i0 < n_items; i0 += 32) {
            const int i = i0 + lane;
            int c = -1, ti = 0;
            real cand = INF, tc = INF;
            uint8_t cset = 0;
            if (i < n_items) {
                c = W.list[i];
                ti = mt_of(c);
                tc = kval(W.kv[ti]);
                const real sp = kHetero ? __ldg(spd + base + c) : (real)spd_const_term;
                if constexpr (kAniso)
                    cand = solve_cell_w<real, kTape>(W.kv, ti, tc, sp, (real)p.wy, (real)p.wz, cset);
                else
                    cand = solve_cell<real, kTape>(W.kv, ti, tc, sp, cset);
            }
            __syncwarp();
            // each cell appears once in the list, so tc is still its value
            if (c >= 0 && lt(cand, tc)) {
                W.kv[ti] = kmark(cand);
                if (kTape)
                    W.tp[c] = cset;
                atomicOr(&W.improved[c & 31], 1u << (c >> 5));
            }
            __syncwarp();
        }
        // a cell whose value dropped is BAND again (Algorithm 10)
        const unsigned imp = W.improved[lane];
        W.improved[lane] = 0u;
        band |= imp;
        known &= ~imp;
        settled &= ~imp;
        pend &= ~imp;
        // minimum of the BAND cells of each side (the heap tops): the cells
        // the last accept scan left plus the cells that just dropped
        real l0 = r0, l1 = r1;
        for (unsigned m = imp; m; m &= m - 1u) {
            const int k = __ffs(m) - 1;
            const real v = kval(W.kv[tb + 40 * (k & 1) + 100 * (k >> 1)]);
            if ((neg >> k) & 1u)
                l0 = vmin(l0, v);
            else
                l1 = vmin(l1, v);
        }
        m0 = warp_min(l0);
        m1 = warp_min(l1);
        if (kMode == 0)
            break;
        if (lt(m0, mp0))
            settled &= ~neg;
        if (lt(m1, mp1))
            settled &= neg;
        mp0 = m0;
        mp1 = m1;
        if (rounds == 0) {
            // cells that were KNOWN when the march began
            for (unsigned m = known & ~settled; m; m &= m - 1u) {
                const int k = __ffs(m) - 1;
                if (!lt((neg >> k) & 1u ? m0 : m1, W.kv[tb + 40 * (k & 1) + 100 * (k >> 1)]))
                    settled |= 1u << k;
            }
        }
        if (!lt(m0, pl0)) {
            settled |= pend & neg;
            pend &= ~neg;
        }
        if (!lt(m1, pl1)) {
            settled |= pend & ~neg;
            pend &= neg;
        }
        // accept the lowest bucket up to the restart bound; the rest give
        // the band minimum of the next round
        const real lim0 = vmin(m0 + delta, bound0), lim1 = vmin(m1 + delta, bound1);
        unsigned acc = 0;
        r0 = INF;
        r1 = INF;
        for (unsigned m = band; m; m &= m - 1u) {
            const int k = __ffs(m) - 1;
            const int ti = tb + 40 * (k & 1) + 100 * (k >> 1);
            const real v = kval(W.kv[ti]);
            const bool ng = (neg >> k) & 1u;
            if (!lt(ng ? lim0 : lim1, v)) {
                acc |= 1u << k;
                W.kv[ti] = v;
            } else if (ng) {
                r0 = vmin(r0, v);
            } else {
                r1 = vmin(r1, v);
            }
        }
        band &= ~acc;
        known |= acc;
        const int nacc = __reduce_add_sync(FULL, (unsigned)__popc(acc));
        if (nacc == 0)
            break;
        acc_any |= acc;
        pend |= acc;
        // a falling minimum lowers lim, so keep the largest lim of the pending cells
        pl0 = lt(pl0, lim0) ? lim0 : pl0;
        pl1 = lt(pl1, lim1) ? lim1 : pl1;
        st.accepted += (unsigned long long)nacc;
        if (++rounds > p.max_rounds) {
            if (lane == 0)
                atomicOr(&s.ctrl->error, ERR_ROUNDS);
            break;
        }
        __syncwarp();
        relax = neighbour_mask(acc, lane) & ~frozen & ~settled;
    }

    // ---- write back, front minima, overlap change notification ------------
    // A boundary cell accepted here (and known at the end) is flagged to the
    // neighbour only if the adjacent halo cell is not known with a value at or
    // below it: such a neighbour cell can never take it as an upwind value
    // (Algorithm 11 uses only smaller known neighbours, and values only
    // decrease), so the exchange would change nothing there.
    unsigned long long fo0 = 0, fo1 = 0, fo2 = 0, fo3 = 0, fo4 = 0, fo5 = 0;
    real fv0 = INF, fv1 = INF;   // smallest flagged value per side
    const unsigned chg = acc_any & known;
    __syncwarp();   // the list buffer holds the tags again from here
#pragma unroll 2
    for (int k = 0; k < 16; ++k) {
        const int c = lane + 32 * k;
        const int ti = tb + 40 * (k & 1) + 100 * (k >> 1);
        const real v = kval(W.kv[ti]);
        uint8_t t;
        if ((out >> k) & 1u)
            t = TG_OUT | ST_FAR;
        else if ((fix >> k) & 1u)
            t = ST_FIX;
        else if ((known >> k) & 1u)
            t = ST_KNOWN;
        else if ((band >> k) & 1u)
            t = ST_BAND;
        else
            t = ST_FAR;
        if ((neg >> k) & 1u)
            t |= TG_NEG;
        stag[c] = t;
        if (kMode == 1 && ((chg >> k) & 1u)) {
            const int y = lr + 4 * (k & 1), z = k >> 1;
            bool flagged = false;
            if (lx == 0 && lt(v, W.kv[ti - 1])) {
                fo0 |= 1ull << (y + 8 * z);
                flagged = true;
            }
            if (lx == 7 && lt(v, W.kv[ti + 1])) {
                fo1 |= 1ull << (y + 8 * z);
                flagged = true;
            }
            if (y == 0 && lt(v, W.kv[ti - kTile])) {
                fo2 |= 1ull << (lx + 8 * z);
                flagged = true;
            }
            if (y == 7 && lt(v, W.kv[ti + kTile])) {
                fo3 |= 1ull << (lx + 8 * z);
                flagged = true;
            }
            if (z == 0 && lt(v, W.kv[ti - kTile * kTile])) {
                fo4 |= 1ull << (lx + 8 * y);
                flagged = true;
            }
            if (z == 7 && lt(v, W.kv[ti + kTile * kTile])) {
                fo5 |= 1ull << (lx + 8 * y);
                flagged = true;
            }
            if (flagged) {
                if ((neg >> k) & 1u)
                    fv0 = vmin(fv0, v);
                else
                    fv1 = vmin(fv1, v);
            }
        }
    }
    // write back with 16-byte stores from the rows of the tile (marks cleared)
    __syncwarp();
    {
        constexpr int kVecs = kB3 * (int)sizeof(real) / 16 / 32;
        uint4 *gv = reinterpret_cast<uint4 *>(T + base);
#pragma unroll
        for (int j = 0; j < kVecs; ++j) {
            const int q = lane + 32 * j;
            gv[q] = row_load(W.kv, q);
        }
        reinterpret_cast<uint4 *>(tag + base)[lane] = reinterpret_cast<const uint4 *>(stag)[lane];
        if (kTape)
            reinterpret_cast<uint4 *>(s.tape + base)[lane] = reinterpret_cast<const uint4 *>(W.tp)[lane];
    }
    notify_v[0] = kMode == 1 ? warp_min(fv0) : INF;
    notify_v[1] = kMode == 1 ? warp_min(fv1) : INF;
    if (lane == 0) {
        bmin[2 * b] = m0;
        bmin[2 * b + 1] = m1;
    }
    notify_m = 0;
    notify_nb = -1;
    if (kMode == 1) {
        unsigned long long m = 0;
#define FMM_FACE_OR(f, val)                                                        \
    {                                                                              \
        const unsigned lo = __reduce_or_sync(FULL, (unsigned)(val));               \
        const unsigned hi = __reduce_or_sync(FULL, (unsigned)((val) >> 32));       \
        if (lane == (f))                                                           \
            m = (unsigned long long)lo | ((unsigned long long)hi << 32);           \
    }
        FMM_FACE_OR(0, fo0) FMM_FACE_OR(1, fo1) FMM_FACE_OR(2, fo2)
        FMM_FACE_OR(3, fo3) FMM_FACE_OR(4, fo4) FMM_FACE_OR(5, fo5)
#undef FMM_FACE_OR
#pragma unroll
        for (int f = 0; f < kFaces; ++f)
            if (lane == f)
                notify_nb = nbi[f];
        notify_m = (lane < kFaces && notify_nb >= 0) ? m : 0ull;
        st.marches += 1;
        st.rounds += (unsigned long long)rounds;
    }
}

__device__ __forceinline__ void flush_stats(Control *ctrl, MarchStats &st, int lane)
{
    const unsigned ex = __reduce_add_sync(FULL, (unsigned)st.exchanges);
    if (lane == 0 && st.marches) {
        atomicAdd(&ctrl->marches, st.marches);
        atomicAdd(&ctrl->rounds, st.rounds);
        atomicAdd(&ctrl->accepted, st.accepted);
        atomicAdd(&ctrl->solves, st.solves);
        atomicAdd(&ctrl->exchanges, (unsigned long long)ex);
    }
}

// Phased march: kMode 0 runs Algorithm 9 over all bricks; kMode 1 runs
// Algorithm 12 over the bricks of work list `which` (taken one at a time from
// a shared counter) with the change masks the select kernel moved to the
// inbox; changes are flagged in the neighbours' live masks and dirty flags.
template <typename real, bool kHetero, int kMode, bool kTape, bool kAniso>
__global__ void __launch_bounds__(kMarchWarps * 32, march_min_blocks<real, kTape>())
    k_march(Geom g, DeviceState s, SolveParams p, double spd_const_term, int which)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpTile<real, kTape> &W = reinterpret_cast<WarpTile<real, kTape> *>(smem_raw)[warp];
    Control *ctrl = s.ctrl;
    if (kMode == 1 && ctrl->done)
        return;
    const long long n = (kMode == 0) ? g.nbricks : (long long)ctrl->n_list[which];
    // select the list without indexing the parameter struct at run time
    // (that would copy the struct to local memory)
    const int *work_list = which ? s.list[1] : s.list[0];
    const real bound0 = (real)ctrl->bound[0], bound1 = (real)ctrl->bound[1];
    MarchStats st = {0, 0, 0, 0, 0};
    long long it = 0, next = 0;
    if (kMode == 1) {
        if (lane == 0) {
            it = (long long)atomicAdd(&ctrl->work[which], 1u);
            next = (long long)atomicAdd(&ctrl->work[which], 1u);
        }
        it = __shfl_sync(FULL, it, 0);
        next = __shfl_sync(FULL, next, 0);
    } else {
        it = (long long)blockIdx.x * kMarchWarps + warp;
    }
    while (it < n) {
        const long long b = (kMode == 0) ? it : (long long)work_list[it];
        if (kMode == 0) {
            // Algorithm 9 only changes cells next to a FIX cell: a brick with
            // no FIX cell in it or in its six neighbours keeps the state of
            // Algorithm 8 and has no BAND cell (one 16-byte load of tags per
            // lane and brick decides)
            bool fixnear = false;
#pragma unroll
            for (int f = -1; f < kFaces; ++f) {
                const long long q = f < 0 ? b : neighbour_brick(g, s.nbr, b, f);
                if (q < 0)
                    continue;
                const uint4 t4 = reinterpret_cast<const uint4 *>(s.tag + q * kB3)[lane];
                const unsigned w = (t4.x & (t4.x >> 1)) | (t4.y & (t4.y >> 1)) | (t4.z & (t4.z >> 1)) |
                                   (t4.w & (t4.w >> 1));
                fixnear = fixnear || (w & 0x01010101u) != 0u;   // a byte with status ST_FIX (3)
            }
            if (!__any_sync(FULL, fixnear)) {
                if (lane < 2)
                    ((real *)s.bmin)[2 * b + lane] = inf_v<real>();
                it += (long long)gridDim.x * kMarchWarps;
                continue;
            }
        }
        unsigned long long F[kFaces];
#pragma unroll
        for (int f = 0; f < kFaces; ++f)
            F[f] = kMode == 1 ? s.inbox[b * kFaces + f] : 0ull;
        unsigned long long m;
        long long nb;
        real nv[2];
        march_brick<real, kHetero, kMode, false, kTape, kAniso>(g, s, p, spd_const_term, W, b, F, bound0, bound1,
                                                 lane, m, nb, nv, st);
        if (kMode == 1 && m) {
            atomicOr(&s.fresh[nb * kFaces + (lane ^ 1)], m);
            s.dirty[nb] = 1u;
            st.exchanges += (unsigned long long)__popcll(m);
        }
        __syncwarp();
        if (kMode == 1) {
            it = next;
            if (it < n && lane == 0)
                next = (long long)atomicAdd(&ctrl->work[which], 1u);
            next = __shfl_sync(FULL, next, 0);
        } else {
            it += (long long)gridDim.x * kMarchWarps;
        }
    }
    if (kMode == 1)
        flush_stats(ctrl, st, lane);
}

// ---------------------------------------------------------------------------
// Persistent restart: one launch marches every brick of a restart to the
// bound until no brick has unconsumed halo changes.  Bricks wait in a ring
// queue; a brick is in the queue or being marched at most once at a time
// (queued[b] = 1 from the push until its march ends), so a brick always has a
// single writer.  A march that changes boundary cells ORs them into the
// neighbour's change masks after a fence and pushes the neighbour if it can
// claim queued[nb]; a brick that ends its march clears queued[b] and pushes
// itself again if masks arrived meanwhile.  `pending` counts bricks pushed and
// not yet done; the launch ends when it reaches zero.  Every wait is bounded:
// past the limit the kernel sets ERR_SPIN and returns.
// ---------------------------------------------------------------------------

template <typename real, bool kHetero, bool kTape, bool kAniso>
__global__ void __launch_bounds__(kMarchWarps * 32, march_min_blocks<real, kTape>())
    k_march_persistent(Geom g, DeviceState s, SolveParams p, double spd_const_term)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpTile<real, kTape> &W = reinterpret_cast<WarpTile<real, kTape> *>(smem_raw)[warp];
    Control *ctrl = s.ctrl;
    if (ctrl->done)
        return;
    const real bound0 = (real)ctrl->bound[0], bound1 = (real)ctrl->bound[1];
    const unsigned long long cap = (unsigned long long)g.nbricks;
    unsigned long long *q = s.queue;
    MarchStats st = {0, 0, 0, 0, 0};
    for (;;) {
        long long b = -1;
        if (lane == 0)
            b = queue_pop(ctrl, q, cap);
        b = __shfl_sync(FULL, b, 0);
        if (b < 0)
            break;
        // take the changes flagged so far (later ones re-queue the brick)
        unsigned long long mine = 0;
        if (lane < kFaces)
            mine = atomicExch(&s.fresh[b * kFaces + lane], 0ull);
        __threadfence();
        unsigned long long F[kFaces];
#pragma unroll
        for (int f = 0; f < kFaces; ++f)
            F[f] = __shfl_sync(FULL, mine, f);
        unsigned long long m;
        long long nb;
        real nv[2];
        march_brick<real, kHetero, 1, true, kTape, kAniso>(g, s, p, spd_const_term, W, b, F, bound0, bound1,
                                            lane, m, nb, nv, st);
        // publish the write-back before flagging anything
        __threadfence();
        __syncwarp();
        if (m) {
            atomicOr(&s.fresh[nb * kFaces + (lane ^ 1)], m);
            st.exchanges += (unsigned long long)__popcll(m);
            // the mask must be visible before the claim: a brick that ends
            // its march clears its flag and then re-reads its masks
            __threadfence();
            if (atomicCAS(&s.queued[nb], 0u, 1u) == 0u) {
                atomicAdd(&ctrl->pending, 1);
                queue_push(ctrl, q, cap, nb);
            }
        }
        __syncwarp();
        if (lane == 0) {
            // end of the march: let neighbours queue the brick again, and do
            // it here if changes arrived while it ran
            atomicExch(&s.queued[b], 0u);
            __threadfence();
            bool again = false;
#pragma unroll
            for (int f = 0; f < kFaces; ++f)
                again = again || (vload(&s.fresh[b * kFaces + f]) != 0ull);
            if (again && atomicCAS(&s.queued[b], 0u, 1u) == 0u) {
                atomicAdd(&ctrl->pending, 1);
                queue_push(ctrl, q, cap, b);
            }
            __threadfence();
            atomicAdd(&ctrl->pending, -1);
        }
        __syncwarp();
    }
    flush_stats(ctrl, st, lane);
}

// ---------------------------------------------------------------------------
// Continuous schedule: the restarts of Algorithm 16 without the barrier
// between them.  One launch marches until the solve is complete.  Each march
// takes the current bound when it starts.  Once fewer bricks than raise_at
// are queued or marching, an idle warp raises the bound to
// max(bound, minimum seen by the last scan) + stride (at most width) and the
// idle warps scan the per-brick minima in chunks, pushing every brick with a
// BAND cell at or below the new bound; a brick that ends a march with a BAND
// cell at or below the current bound pushes itself again.  The bricks of the
// last shell of one restart thus overlap the first bricks of the next.  epoch
// works as a sequence lock: odd while a raise rewrites the bound and the scan
// counters.  The solve is complete when no raise is in progress, the last
// scan is done, nothing is queued or marching and the bound has reached width
// on both sides.  At the restart limit the raises stop and the launch ends
// once the current level is drained, so the solve can be resumed from there.
// Every wait is bounded (wait_ns without any progress).
// ---------------------------------------------------------------------------

__device__ __forceinline__ double vloadd(const double *p) { return *(const volatile double *)p; }
__device__ __forceinline__ unsigned long long vloadu(const unsigned long long *p)
{
    return *(const volatile unsigned long long *)p;
}

// Push, with one tail increment for the warp, the bricks b of the lanes whose
// sel is set and that claim queued[b].
__device__ __forceinline__ void queue_push_warp(Control *c, unsigned long long *q, unsigned long long cap,
                                                unsigned *queued, long long b, bool sel, int lane)
{
    const bool mine = sel && atomicCAS(&queued[b], 0u, 1u) == 0u;
    const unsigned ball = __ballot_sync(FULL, mine);
    if (ball == 0u)
        return;
    unsigned long long t0 = 0;
    if (lane == 0) {
        atomicAdd(&c->pending, __popc(ball));
        t0 = atomicAdd(&c->q_tail, (unsigned long long)__popc(ball));
    }
    t0 = __shfl_sync(FULL, t0, 0);
    if (mine) {
        const unsigned long long t = t0 + __popc(ball & ((1u << lane) - 1u));
        const unsigned long long v = ((t & 0xffffffffull) << 32) | (unsigned long long)(b + 1);
        unsigned long long *slot = q + (t % cap);
        const unsigned long long ts = device_ns(), lim = vload(&c->wait_ns);
        while (atomicCAS(slot, 0ull, v) != 0ull) {
            if (device_ns() - ts > lim || (vload((const int *)&c->error) & ERR_SPIN)) {
                atomicOr(&c->error, ERR_SPIN);
                break;
            }
            __nanosleep(32);
        }
    }
}

// The smallest value neighbours flagged to brick side j (2 b + side) since it
// last took its masks, +inf when none is recorded.
constexpr unsigned long long kInminNone = ~0ull;
template <typename real>
__device__ __forceinline__ real inmin_bits(unsigned long long v)
{
    return v >= 0x7ff0000000000000ull ? inf_v<real>() : (real)__longlong_as_double((long long)v);
}
// both BAND minima of a brick (adjacent, 16- or 8-byte aligned) in one load
__device__ __forceinline__ void ld_pair(const double *p, double &a, double &b)
{
    const double2 v = __ldcg(reinterpret_cast<const double2 *>(p));
    a = v.x;
    b = v.y;
}
__device__ __forceinline__ void ld_pair(const float *p, float &a, float &b)
{
    const float2 v = __ldcg(reinterpret_cast<const float2 *>(p));
    a = v.x;
    b = v.y;
}

template <typename real>
__device__ __forceinline__ real inmin_value(const unsigned long long *inmin, long long j)
{
    const unsigned long long v = vloadu(inmin + j);
    return v >= 0x7ff0000000000000ull ? inf_v<real>() : (real)__longlong_as_double((long long)v);
}

// One warp scans chunk ch of the per-brick minima for the bound (bd0, bd1).
template <typename real>
__device__ __forceinline__ void scan_chunk(const Geom &g, const DeviceState &s, int ch, real bd0,
                                           real bd1, int lane)
{
    Control *c = s.ctrl;
    const real *bmin = (const real *)s.bmin;
    const real INF = inf_v<real>();
    const unsigned long long cap = (unsigned long long)g.nbricks;
    real l0 = INF, l1 = INF;
    const long long first = (long long)ch * kScanChunk;
    // kScanBatch bricks per lane at a time: both minima of a brick in one
    // load, both flagged values in another, all loads of a batch in flight
    // together (the scan is a chain of L2 round trips otherwise)
    constexpr int kScanBatch = 2;
    static_assert((kScanChunk / 32) % kScanBatch == 0, "whole batches per chunk");
    for (int j0 = 0; j0 < kScanChunk / 32; j0 += kScanBatch) {
        real bm[kScanBatch][2];
        ulonglong2 im[kScanBatch];
#pragma unroll
        for (int u = 0; u < kScanBatch; ++u) {
            const long long b = first + 32 * (j0 + u) + lane;
            if (b < g.nbricks) {
                ld_pair(bmin + 2 * b, bm[u][0], bm[u][1]);
                im[u] = __ldcg(reinterpret_cast<const ulonglong2 *>(s.inmin + 2 * b));
            } else {
                bm[u][0] = bm[u][1] = INF;
                im[u] = make_ulonglong2(kInminNone, kInminNone);
            }
        }
#pragma unroll
        for (int u = 0; u < kScanBatch; ++u) {
            const long long b = first + 32 * (j0 + u) + lane;
            const real m0 = vmin(bm[u][0], inmin_bits<real>(im[u].x));
            const real m1 = vmin(bm[u][1], inmin_bits<real>(im[u].y));
            l0 = vmin(l0, m0);
            l1 = vmin(l1, m1);
            const bool sel = b < g.nbricks && ((lt(m0, INF) && !lt(bd0, m0)) || (lt(m1, INF) && !lt(bd1, m1)));
            queue_push_warp(c, s.queue, cap, s.queued, b, sel, lane);
        }
    }
    l0 = warp_min(l0);
    l1 = warp_min(l1);
    if (lane == 0) {
        atomicMin(&c->scan_min[0], (unsigned long long)__double_as_longlong((double)l0));
        atomicMin(&c->scan_min[1], (unsigned long long)__double_as_longlong((double)l1));
        __threadfence();
        atomicAdd(&c->scan_done, 1);
    }
}

// Raise the bound (lane 0).  Returns true when this warp raised it.  For each
// side, with m the smallest BAND minimum the last scan saw, the new bound is
// max(bound, m) + stride, but while bricks are queued or marching at most
// max_lead strides above floor(m / stride) * stride, so a small front
// cannot run ahead.  A scan that saw no BAND cell on a side proves the side
// finished only if it started with nothing queued or marching (a clean
// scan): otherwise the side's next BAND cells may have been in flight, in
// bricks notified but not yet marched, and the side waits while bricks are
// in flight, or rises by one stride (which starts a clean scan) when none
// are.  With nothing queued or marching every BAND value is above the
// bound, so the bound always rises.
__device__ bool try_raise(Control *c, const SolveParams &p, int nchunks, int pend)
{
    const int e = vload(&c->epoch);
    if ((e & 1) || vload(&c->scan_done) < nchunks)
        return false;
    const double b0 = vloadd(&c->bound[0]), b1 = vloadd(&c->bound[1]);
    if (b0 >= p.width && b1 >= p.width)
        return false;
    double nb[2];
    const double bo[2] = {b0, b1};
#pragma unroll
    for (int sd = 0; sd < 2; ++sd) {
        const double sm = __longlong_as_double((long long)vloadu(&c->scan_min[sd]));
        double v;
        if (!(sm < CUDART_INF)) {
            if (pend > 0)
                v = bo[sd];
            else if (vload(&c->scan_clean))
                v = p.width;
            else
                v = fmin(bo[sd] + p.stride, p.width);
        } else {
            v = fmax(bo[sd], sm) + p.stride;
            if (pend > 0 && p.stride < CUDART_INF)
                v = fmin(v, (floor(sm / p.stride) + p.max_lead) * p.stride);
            v = fmin(v, p.width);
        }
        nb[sd] = fmax(v, bo[sd]);
    }
    if (!(nb[0] > b0 || nb[1] > b1))
        return false;
    if (atomicCAS(&c->epoch, e, e + 1) != e)
        return false;
    if (p.max_restarts > 0 && (long long)vload(&c->restart) >= p.max_restarts) {
        // the restart limit counts the raises too
        atomicOr(&c->error, ERR_RESTARTS);
        __threadfence();
        atomicExch(&c->epoch, e + 2);
        return false;
    }
    atomicExch(&c->scan_done, 0);
    atomicExch(&c->scan_clean, pend == 0 ? 1 : 0);
    __threadfence();
    *(volatile double *)&c->bound[0] = nb[0];
    *(volatile double *)&c->bound[1] = nb[1];
    atomicExch(&c->scan_min[0], 0x7ff0000000000000ull);
    atomicExch(&c->scan_min[1], 0x7ff0000000000000ull);
    atomicAdd(&c->restart, 1);
    __threadfence();
    atomicExch(&c->scan_next, 0);
    __threadfence();
    atomicExch(&c->epoch, e + 2);
    return true;
}

// The solve is complete (lane 0; see above).
// The launch ends when the solve is complete or, once the restart limit has
// stopped the raises (limited), when the current level is drained: no raise
// or scan in progress and nothing queued or marching.  The state is then the
// one after a restart of Algorithm 16, from which a solve can resume.
__device__ bool launch_done(Control *c, const SolveParams &p, int nchunks, bool limited)
{
    const int e = vload(&c->epoch);
    if ((e & 1) || vload(&c->scan_done) < nchunks)
        return false;
    __threadfence();
    if (vload(&c->pending) != 0)
        return false;
    if (!limited && (vloadd(&c->bound[0]) < p.width || vloadd(&c->bound[1]) < p.width))
        return false;
    __threadfence();
    return vload(&c->epoch) == e;
}

// Lane 0: the next job of the warp.  job 0: march brick arg; 1: scan chunk
// arg; 2: stop.  ticket is the queue ticket the warp holds (-1: none).
__device__ void next_job(Control *c, unsigned long long *q, unsigned long long cap,
                         const SolveParams &p, int nchunks, long long &ticket, int &job,
                         long long &arg)
{
    if (ticket < 0)
        ticket = (long long)atomicAdd(&c->q_head, 1ull);
    unsigned long long *slot = q + ((unsigned long long)ticket % cap);
    const unsigned long long want = (unsigned long long)ticket & 0xffffffffull;
    unsigned long long t0 = device_ns();
    unsigned long long seen_tail = vloadu(&c->q_tail);
    const unsigned long long lim = vloadu(&c->wait_ns);
    int seen_done = vload(&c->scan_done), seen_epoch = vload(&c->epoch);
    unsigned ns = 64;
    for (;;) {
        const unsigned long long v = vloadu(slot);
        if (v != 0ull && (v >> 32) == want) {
            atomicExch(slot, 0ull);
            ticket = -1;
            job = 0;
            arg = (long long)(v & 0xffffffffull) - 1;
            return;
        }
        const int err = vload(&c->error);
        if (err & ERR_SPIN) {
            job = 2;
            return;
        }
        const bool limited = (err & ERR_RESTARTS) != 0;
        if (vload(&c->scan_next) < nchunks) {
            const int ch = atomicAdd(&c->scan_next, 1);
            if (ch < nchunks) {
                job = 1;
                arg = ch;
                return;
            }
        }
        const int pend = vload(&c->pending);
        if (!limited && pend < p.raise_at && try_raise(c, p, nchunks, pend))
            continue;
        if (pend == 0 && launch_done(c, p, nchunks, limited)) {
            job = 2;
            return;
        }
        const unsigned long long now = device_ns(), tail = vloadu(&c->q_tail);
        const int dn = vload(&c->scan_done), ep = vload(&c->epoch);
        if (tail != seen_tail || dn != seen_done || ep != seen_epoch) {
            seen_tail = tail;
            seen_done = dn;
            seen_epoch = ep;
            t0 = now;
        } else if (now - t0 > lim) {
            break;
        }
        __nanosleep(ns);
        if (ns < 2048)
            ns <<= 1;
    }
    atomicOr(&c->error, ERR_SPIN);
    job = 2;
}

template <typename real, bool kHetero, bool kTape, bool kAniso>
__global__ void __launch_bounds__(kMarchWarps * 32, march_min_blocks<real, kTape>())
    k_march_continuous(Geom g, DeviceState s, SolveParams p, double spd_const_term)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpTile<real, kTape> &W = reinterpret_cast<WarpTile<real, kTape> *>(smem_raw)[warp];
    Control *ctrl = s.ctrl;
    if (ctrl->done)
        return;
    const unsigned long long cap = (unsigned long long)g.nbricks;
    const int nchunks = (int)((g.nbricks + kScanChunk - 1) / kScanChunk);
    const real *bmin = (const real *)s.bmin;
    unsigned long long *q = s.queue;
    MarchStats st = {0, 0, 0, 0, 0};
    long long ticket = -1;
    for (;;) {
        int job = 2;
        long long arg = 0;
        if (lane == 0)
            next_job(ctrl, q, cap, p, nchunks, ticket, job, arg);
        job = __shfl_sync(FULL, job, 0);
        arg = __shfl_sync(FULL, arg, 0);
        if (job == 2)
            break;
        if (job == 1) {
            real bd0 = 0, bd1 = 0;
            if (lane == 0) {
                bd0 = (real)vloadd(&ctrl->bound[0]);
                bd1 = (real)vloadd(&ctrl->bound[1]);
            }
            bd0 = __shfl_sync(FULL, bd0, 0);
            bd1 = __shfl_sync(FULL, bd1, 0);
            scan_chunk<real>(g, s, (int)arg, bd0, bd1, lane);
            continue;
        }
        const long long b = arg;
        // forget the smallest flagged value, then take the masks: a value
        // flagged in between is lost, and a brick with masks but no value
        // counts as ready (below)
        if (lane < 2)
            atomicExch(&s.inmin[2 * b + lane], kInminNone);
        __threadfence();
        __syncwarp();
        unsigned long long mine = 0;
        if (lane < kFaces)
            mine = atomicExch(&s.fresh[b * kFaces + lane], 0ull);
        real bound0 = 0, bound1 = 0;
        if (lane == 0) {
            // accept up to the bound plus the look-ahead, never beyond
            // width_band (cells above it stay BAND, Algorithm 12)
            bound0 = (real)fmin(vloadd(&ctrl->bound[0]) + p.ahead, p.width);
            bound1 = (real)fmin(vloadd(&ctrl->bound[1]) + p.ahead, p.width);
        }
        __threadfence();
        bound0 = __shfl_sync(FULL, bound0, 0);
        bound1 = __shfl_sync(FULL, bound1, 0);
        unsigned long long F[kFaces];
#pragma unroll
        for (int f = 0; f < kFaces; ++f)
            F[f] = __shfl_sync(FULL, mine, f);
        unsigned long long m;
        long long nb;
        real nv[2];
        march_brick<real, kHetero, 1, true, kTape, kAniso>(g, s, p, spd_const_term, W, b, F, bound0, bound1,
                                            lane, m, nb, nv, st);
        __threadfence();
        __syncwarp();
        if (m) {
            // the value first, then the mask: a brick that sees the mask
            // also sees a value at most this one (or none, see above)
            const real INF = inf_v<real>();
            if (lt(nv[0], INF))
                atomicMin(&s.inmin[2 * nb], (unsigned long long)__double_as_longlong((double)nv[0]));
            if (lt(nv[1], INF))
                atomicMin(&s.inmin[2 * nb + 1], (unsigned long long)__double_as_longlong((double)nv[1]));
            __threadfence();
            atomicOr(&s.fresh[nb * kFaces + (lane ^ 1)], m);
            st.exchanges += (unsigned long long)__popcll(m);
            __threadfence();
            // the neighbour starts now if what it was sent is at or below
            // the bound; otherwise the scan of a later bound pushes it
            const real cb0 = (real)vloadd(&ctrl->bound[0]), cb1 = (real)vloadd(&ctrl->bound[1]);
            const bool ready = (lt(nv[0], INF) && !lt(cb0, nv[0])) || (lt(nv[1], INF) && !lt(cb1, nv[1]));
            if (ready && atomicCAS(&s.queued[nb], 0u, 1u) == 0u) {
                atomicAdd(&ctrl->pending, 1);
                queue_push(ctrl, q, cap, nb);
            }
        }
        __syncwarp();
        if (lane == 0) {
            const real INF = inf_v<real>();
            const real m0 = bmin[2 * b], m1 = bmin[2 * b + 1];
            // end of the march: let others queue the brick again, and do it
            // here if changes at or below the bound arrived meanwhile (or
            // changes without a recorded value) or the bound has risen above
            // one of its BAND minima
            atomicExch(&s.queued[b], 0u);
            __threadfence();
            bool flagged = false;
#pragma unroll
            for (int f = 0; f < kFaces; ++f)
                flagged = flagged || (vload(&s.fresh[b * kFaces + f]) != 0ull);
            const real nb0 = (real)vloadd(&ctrl->bound[0]), nb1 = (real)vloadd(&ctrl->bound[1]);
            bool again = false;
            if (flagged) {
                const unsigned long long i0 = vloadu(&s.inmin[2 * b]), i1 = vloadu(&s.inmin[2 * b + 1]);
                const real v0 = inmin_value<real>(s.inmin, 2 * b), v1 = inmin_value<real>(s.inmin, 2 * b + 1);
                again = (i0 == kInminNone && i1 == kInminNone) || (lt(v0, INF) && !lt(nb0, v0)) ||
                        (lt(v1, INF) && !lt(nb1, v1));
            }
            again = again || (lt(m0, INF) && !lt(nb0, m0)) || (lt(m1, INF) && !lt(nb1, m1));
            if (again && atomicCAS(&s.queued[b], 0u, 1u) == 0u) {
                atomicAdd(&ctrl->pending, 1);
                queue_push(ctrl, q, cap, b);
            }
            __threadfence();
            atomicAdd(&ctrl->pending, -1);
        }
        __syncwarp();
    }
    flush_stats(ctrl, st, lane);
}

// Seed the queue of a restart: bricks with a BAND cell at or below the bound.
template <typename real>
__global__ void k_seed(Geom g, const real *__restrict__ bmin, const unsigned long long *inmin,
                       Control *ctrl, unsigned *queued, unsigned long long *q)
{
    if (ctrl->done)
        return;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        // no scan in progress (the continuous schedule raises the bound later)
        const int nchunks = (int)((g.nbricks + kScanChunk - 1) / kScanChunk);
        ctrl->epoch = 0;
        ctrl->scan_next = nchunks;
        ctrl->scan_done = nchunks;
        ctrl->scan_clean = 0;
        if (ctrl->hold)
            atomicAdd(&ctrl->pending, 1);   // testing: the queue never drains
        // as if a scan had seen the bound itself: the first raise adds one stride
        ctrl->scan_min[0] = (unsigned long long)__double_as_longlong(ctrl->bound[0]);
        ctrl->scan_min[1] = (unsigned long long)__double_as_longlong(ctrl->bound[1]);
    }
    const double bd0 = ctrl->bound[0], bd1 = ctrl->bound[1];
    const int lane = threadIdx.x & 31;
    for (long long b0 = blockIdx.x * (long long)blockDim.x; b0 < g.nbricks;
         b0 += (long long)gridDim.x * blockDim.x) {
        const long long b = b0 + threadIdx.x;
        bool sel = false;
        if (b < g.nbricks) {
            const double m0 = fmin((double)bmin[2 * b], inmin_value<double>(inmin, 2 * b));
            const double m1 = fmin((double)bmin[2 * b + 1], inmin_value<double>(inmin, 2 * b + 1));
            sel = (m0 < CUDART_INF && m0 <= bd0) || (m1 < CUDART_INF && m1 <= bd1);
        }
        const unsigned ball = __ballot_sync(0xffffffffu, sel);
        if (ball == 0u)
            continue;
        unsigned long long basepos = 0;
        if (lane == 0) {
            basepos = atomicAdd(&ctrl->q_tail, (unsigned long long)__popc(ball));
            atomicAdd(&ctrl->pending, __popc(ball));
        }
        basepos = __shfl_sync(0xffffffffu, basepos, 0);
        if (sel) {
            const unsigned long long t = basepos + __popc(ball & ((1u << lane) - 1u));
            queued[b] = 1u;
            q[t % (unsigned long long)g.nbricks] = ((t & 0xffffffffull) << 32) | (unsigned long long)(b + 1);
        }
    }
}

// ---------------------------------------------------------------------------
// Algorithm 16 bookkeeping: global minima of the front, exit test, bound.
// ---------------------------------------------------------------------------

template <typename real>
__global__ void k_reduce(Geom g, const real *__restrict__ bmin, const unsigned long long *inmin,
                         const unsigned *__restrict__ dirty, Control *ctrl)
{
    if (ctrl->done)
        return;
    __shared__ double r0[8], r1[8];
    __shared__ unsigned rc[8];
    double m0 = CUDART_INF, m1 = CUDART_INF;
    unsigned cnt = 0;
    for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b < g.nbricks;
         b += (long long)gridDim.x * blockDim.x) {
        m0 = fmin(m0, fmin((double)bmin[2 * b], inmin_value<double>(inmin, 2 * b)));
        m1 = fmin(m1, fmin((double)bmin[2 * b + 1], inmin_value<double>(inmin, 2 * b + 1)));
        cnt += dirty[b] != 0u;
    }
    m0 = warp_min(m0);
    m1 = warp_min(m1);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        r0[w] = m0;
        r1[w] = m1;
        rc[w] = cnt;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < (int)(blockDim.x >> 5); ++i) {
            m0 = fmin(m0, r0[i]);
            m1 = fmin(m1, r1[i]);
            cnt += rc[i];
        }
        atomicMin(&ctrl->minbits[0], (unsigned long long)__double_as_longlong(m0));
        atomicMin(&ctrl->minbits[1], (unsigned long long)__double_as_longlong(m1));
        if (cnt)
            atomicAdd(&ctrl->dirty_count, cnt);
    }
}

__global__ void k_control(Control *c, double width, double stride, long long max_restarts)
{
    if (c->done)
        return;
    if (c->error & (ERR_SPIN | ERR_ROUNDS | ERR_RESTARTS)) {
        c->done = 1;   // a device error ends the solve (reported by the host)
        return;
    }
    const unsigned long long INF_BITS = 0x7ff0000000000000ull;
    double mv0 = fmin(__longlong_as_double((long long)c->minbits[0]), width);
    double mv1 = fmin(__longlong_as_double((long long)c->minbits[1]), width);
    c->restart += 1;
    c->host_restart += 1;
    if (mv0 >= width && mv1 >= width && c->dirty_count == 0u) {
        c->done = 1;
    } else if (max_restarts > 0 && c->restart > max_restarts) {
        c->error |= ERR_RESTARTS;
        c->done = 1;
    } else {
        c->bound[0] = fmin(mv0 + stride, width);
        c->bound[1] = fmin(mv1 + stride, width);
    }
    c->minbits[0] = INF_BITS;
    c->minbits[1] = INF_BITS;
    c->dirty_count = 0u;
    c->n_list[0] = 0u;
    c->n_list[1] = 0u;
    c->work[0] = 0u;
    c->work[1] = 0u;
    c->q_head = 0ull;
    c->q_tail = 0ull;
    c->pending = 0;
}

// Work lists: list 0 = bricks with a BAND cell at or below the bound or with
// pending overlap changes (first march); list 1 = bricks with pending changes
// (second march, after the exchange).  A selected brick's change masks are
// moved to its inbox here, between kernels, so the march reads them without
// atomics; changes flagged during the march accumulate in the live masks for
// the next selection.
template <typename real>
__global__ void k_select(Geom g, const real *__restrict__ bmin, unsigned *dirty,
                         unsigned long long *fresh, unsigned long long *inbox, Control *ctrl,
                         int *list, int which)
{
    if (ctrl->done)
        return;
    const double bd0 = ctrl->bound[0], bd1 = ctrl->bound[1];
    const int lane = threadIdx.x & 31;
    for (long long b0 = blockIdx.x * (long long)blockDim.x; b0 < g.nbricks;
         b0 += (long long)gridDim.x * blockDim.x) {
        const long long b = b0 + threadIdx.x;
        bool sel = false, dty = false;
        if (b < g.nbricks) {
            dty = dirty[b] != 0u;
            sel = dty;
            if (which == 0) {
                // a brick takes part when it has a BAND cell at or below the
                // bound (an empty side has bound +inf, and so do the minima
                // of bricks without BAND cells)
                const double m0 = (double)bmin[2 * b], m1 = (double)bmin[2 * b + 1];
                sel = sel || (m0 < CUDART_INF && m0 <= bd0) || (m1 < CUDART_INF && m1 <= bd1);
            }
        }
        if (sel) {
#pragma unroll
            for (int f = 0; f < kFaces; ++f) {
                inbox[b * kFaces + f] = dty ? fresh[b * kFaces + f] : 0ull;
                if (dty)
                    fresh[b * kFaces + f] = 0ull;
            }
            if (dty)
                dirty[b] = 0u;
        }
        const unsigned ball = __ballot_sync(0xffffffffu, sel);
        if (ball == 0u)
            continue;
        unsigned basepos = 0;
        if (lane == 0)
            basepos = atomicAdd(&ctrl->n_list[which], (unsigned)__popc(ball));
        basepos = __shfl_sync(0xffffffffu, basepos, 0);
        if (sel)
            list[basepos + __popc(ball & ((1u << lane) - 1u))] = (int)b;
    }
}

__global__ void k_reset_control(Control *c, unsigned long long wait_ns, int hold)
{
    c->wait_ns = wait_ns;
    c->hold = hold;
    const unsigned long long INF_BITS = 0x7ff0000000000000ull;
    c->minbits[0] = INF_BITS;
    c->minbits[1] = INF_BITS;
    c->marches = c->rounds = c->exchanges = c->accepted = c->solves = 0ull;
    c->bound[0] = c->bound[1] = 0.0;
    c->dirty_count = 0u;
    c->n_list[0] = c->n_list[1] = 0u;
    c->work[0] = c->work[1] = 0u;
    c->q_head = c->q_tail = 0ull;
    c->pending = 0;
    c->done = 0;
    c->error = 0;
    c->restart = 0;
    c->host_restart = 0;
    c->epoch = 0;
}

// Brick layout -> the caller's x-fastest arrays (signed psi, public tags);
// one CTA per brick, each warp writing rows of 8 consecutive cells.
template <typename real>
__global__ void __launch_bounds__(kInitThreads) k_output(Geom g, const real *__restrict__ T,
                                                         const uint8_t *__restrict__ tag, real *T_out,
                                                         uint8_t *tags_out)
{
    static_assert(kB3 == 2 * kInitThreads, "two cells per thread");
    for (int b = blockIdx.x; b < (int)g.nbricks; b += gridDim.x) {
        int bx, by, bz;
        brick_xyz32(g, b, bx, by, bz);
        const long long base = (long long)b * kB3;
        // cells c and c + 256 of the brick (z and z + 4), both loaded first
        const int c = threadIdx.x;
        const real v0 = T[base + c], v1 = T[base + c + kInitThreads];
        const uint8_t t0 = tag[base + c], t1 = tag[base + c + kInitThreads];
        const int i = bx * kB + (c & 7), j = by * kB + ((c >> 3) & 7), k = bz * kB + (c >> 6);
        if (i >= g.nx || j >= g.ny)
            continue;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int kk = k + 4 * h;
            if (kk >= g.nz)
                continue;
            const real v = h ? v1 : v0;
            const uint8_t tg = h ? t1 : t0;
            const uint8_t st = tg & ST_MASK;
            // the sign as a bit (a double negation would take the FP64 pipe)
            const real out = st == ST_FAR ? inf_v<real>() : ((tg & TG_NEG) ? kmark(v) : v);
            const long long p = ((long long)kk * g.ny + j) * g.nx + i;
            T_out[p] = out;
            if (tags_out)
                tags_out[p] = st;
        }
    }
}

// ---------------------------------------------------------------------------
// Domain decomposition (Sec. 4.1, Algorithms 13-15): the grid of one rank is
// its slab of z layers plus the ghost layers it shares with its neighbours;
// the overlap layers are read out (signed psi, +inf for FAR cells) and the
// neighbour's copy of them is integrated.
// ---------------------------------------------------------------------------

template <typename real>
__global__ void k_layer_export(Geom g, const real *__restrict__ T, const uint8_t *__restrict__ tag,
                               int z0, int nl, real *out)
{
    const long long n = (long long)g.nx * g.ny * nl;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(p % g.nx);
        const long long r = p / g.nx;
        const int j = (int)(r % g.ny), k = z0 + (int)(r / g.ny);
        const long long b = ((long long)(k >> 3) * g.nby + (j >> 3)) * g.nbx + (i >> 3);
        const long long e = b * kB3 + (i & 7) + 8 * (j & 7) + 64 * (k & 7);
        const uint8_t tg = tag[e];
        real v = T[e];
        if ((tg & ST_MASK) == ST_FAR)
            v = inf_v<real>();
        else if (tg & TG_NEG)
            v = -v;
        out[p] = v;
    }
}

// Algorithm 15: a received value smaller in magnitude than the local one
// replaces it; the cell becomes BAND of the received value's side, so the
// next march accepts it if it is within the bound (KNOWN_OLD of Algorithm
// 15, then taken from the heap) or keeps it tentative (BAND_OLD).  FIX
// cells are never replaced.  count receives the number of replaced cells.
template <typename real>
__global__ void k_layer_integrate(Geom g, real *T, uint8_t *tag, real *bmin, int z0, int nl,
                                  const real *__restrict__ in, unsigned *count)
{
    const long long n = (long long)g.nx * g.ny * nl;
    unsigned c = 0;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(p % g.nx);
        const long long r = p / g.nx;
        const int j = (int)(r % g.ny), k = z0 + (int)(r / g.ny);
        const long long b = ((long long)(k >> 3) * g.nby + (j >> 3)) * g.nbx + (i >> 3);
        const long long e = b * kB3 + (i & 7) + 8 * (j & 7) + 64 * (k & 7);
        const real v = in[p];
        const real a = kval(v);   // |v|, -0 included
        const uint8_t tg = tag[e];
        if ((tg & ST_MASK) == ST_FIX || !(a < inf_v<real>()))
            continue;
        const bool far = (tg & ST_MASK) == ST_FAR;
        if (!far && !lt(a, T[e]))
            continue;
        const bool neg = v < (real)0 || (v == (real)0 && (tg & TG_NEG));
        T[e] = a;
        tag[e] = (uint8_t)(ST_BAND | (neg ? TG_NEG : 0));
        if constexpr (sizeof(real) == 8)
            atomicMin((unsigned long long *)&bmin[2 * b + (neg ? 0 : 1)],
                      (unsigned long long)__double_as_longlong(a));
        else
            atomicMin((unsigned *)&bmin[2 * b + (neg ? 0 : 1)], __float_as_uint(a));
        ++c;
    }
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0 && c)
        atomicAdd(count, c);
}

// Set the bound of a march to a given level (both sides) and empty the queue.
__global__ void k_set_bound(Control *c, double b0, double b1)
{
    c->bound[0] = b0;
    c->bound[1] = b1;
    c->done = 0;
    c->q_head = 0ull;
    c->q_tail = 0ull;
    c->pending = 0;
    c->minbits[0] = c->minbits[1] = 0x7ff0000000000000ull;
    c->dirty_count = 0u;
}

// ---------------------------------------------------------------------------
// Batches: the bricks of many grids packed into one brick array.  bgrid[b] is
// the grid of brick b; the grid table gives its size, first brick, spacing
// and the caller's arrays.  The neighbour table (DeviceState::nbr) has no
// neighbour across the border of a grid, so the grids never exchange data.
// ---------------------------------------------------------------------------

__device__ __forceinline__ void batch_cell(const BatchGrid &G, long long b, int c, int &i, int &j,
                                           int &k)
{
    // a batch has fewer than 2^31 bricks: 32-bit arithmetic
    const int lb = (int)(b - G.brick0);
    const int bx = lb % G.nbx;
    const int r = lb / G.nbx;
    const int by = r % G.nby, bz = r / G.nby;
    i = bx * kB + (c & 7);
    j = by * kB + ((c >> 3) & 7);
    k = bz * kB + (c >> 6);
}

// Algorithm 8 for every grid of a batch: a grid with a level set gets its
// interface cells (reinit_cell), a grid of point sources starts all FAR
// (k_batch_sources then fixes its sources).
template <typename real>
__global__ void k_batch_init(const BatchGrid *__restrict__ grids, const int *__restrict__ bgrid,
                             long long nbricks, real *T, uint8_t *tag)
{
    const long long n = nbricks * kB3;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const long long b = e >> 9;
        const BatchGrid &G = grids[bgrid[b]];
        int i, j, k;
        batch_cell(G, b, (int)(e & 511), i, j, k);
        if (i >= G.nx || j >= G.ny || k >= G.nz) {
            T[e] = inf_v<real>();
            tag[e] = TG_OUT | ST_FAR;
            continue;
        }
        if (!G.phi0) {
            T[e] = inf_v<real>();
            tag[e] = ST_FAR;
            continue;
        }
        real Tv;
        uint8_t tg;
        reinit_cell<real>((const real *)G.phi0, G.nx, G.ny, G.nz, i, j, k, G.h, G.h, G.h, Tv, tg);
        T[e] = Tv;
        tag[e] = tg;
    }
}

// The point sources of the batch: psi = 0, FIX (Algorithm 8).
template <typename real>
__global__ void k_batch_sources(const BatchGrid *__restrict__ grids, const long long *__restrict__ src,
                                long long n_src, real *T, uint8_t *tag)
{
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n_src;
         s += (long long)gridDim.x * blockDim.x) {
        const BatchGrid &G = grids[src[4 * s]];
        const int i = (int)src[4 * s + 1], j = (int)src[4 * s + 2], k = (int)src[4 * s + 3];
        const long long b = G.brick0 + ((long long)(k >> 3) * G.nby + (j >> 3)) * G.nbx + (i >> 3);
        const long long e = b * kB3 + (i & 7) + 8 * (j & 7) + 64 * (k & 7);
        T[e] = (real)0;
        tag[e] = ST_FIX;
    }
}

// Speed term (h_g/F)^2 of every cell of a batch (each grid its own h and its
// own speed field or constant) and the bucket width h_g min(1/F) / sqrt(3)
// of every brick; one CTA of 512 threads per brick, as k_load_speed.
template <typename real>
__global__ void __launch_bounds__(kThreads) k_batch_speed(const BatchGrid *__restrict__ grids,
                                                          const int *__restrict__ bgrid,
                                                          long long nbricks, real *spd, real *bdelta,
                                                          Control *ctrl)
{
    __shared__ real red[kThreads / 32];
    const int t = threadIdx.x;
    for (long long b = blockIdx.x; b < nbricks; b += gridDim.x) {
        const BatchGrid &G = grids[bgrid[b]];
        int i, j, k;
        batch_cell(G, b, t, i, j, k);
        const bool out = i >= G.nx || j >= G.ny || k >= G.nz;
        real F = (real)G.speed_const;
        if (G.speed && !out)
            F = ((const real *)G.speed)[((long long)k * G.ny + j) * G.nx + i];
        if (out)
            F = (real)1;
        if (!(F >= (real)0) || !(F < inf_v<real>()))
            atomicOr(&ctrl->error, ERR_SPEED);
        spd[b * kB3 + t] = speed_term(F, G.h);
        real fm = out ? (real)0 : F;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            fm = fmax(fm, __shfl_xor_sync(0xffffffffu, fm, o));
        if ((t & 31) == 0)
            red[t >> 5] = fm;
        __syncthreads();
        if (t == 0) {
            real mx = red[0];
            for (int w = 1; w < kThreads / 32; ++w)
                mx = fmax(mx, red[w]);
            if (!(mx > (real)0))
                mx = (real)1;
            bdelta[b] = (real)(G.h / (1.7320508075688772 * (double)mx));
        }
        __syncthreads();
    }
}

template <typename real>
__global__ void k_batch_output(const BatchGrid *__restrict__ grids, const int *__restrict__ bgrid,
                               long long nbricks, const real *__restrict__ T,
                               const uint8_t *__restrict__ tag)
{
    const long long n = nbricks * kB3;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const long long b = e >> 9;
        const BatchGrid &G = grids[bgrid[b]];
        int i, j, k;
        batch_cell(G, b, (int)(e & 511), i, j, k);
        if (i >= G.nx || j >= G.ny || k >= G.nz)
            continue;
        const long long p = ((long long)k * G.ny + j) * G.nx + i;
        const real v = T[e];
        const uint8_t tg = tag[e];
        const uint8_t st = tg & ST_MASK;
        real out = v;
        if (st == ST_FAR)
            out = inf_v<real>();
        else if (tg & TG_NEG)
            out = -v;
        ((real *)G.T_out)[p] = out;
        if (G.tags_out)
            G.tags_out[p] = st;
    }
}

int grid_for(long long n, int threads, int cap)
{
    long long b = (n + threads - 1) / threads;
    if (b < 1)
        b = 1;
    if (b > cap)
        b = cap;
    return (int)b;
}

template <typename real, bool kTape>
size_t march_smem() { return sizeof(WarpTile<real, kTape>) * kMarchWarps; }

// Deterministic mode: face f of brick b is its boundary layer on side f
// (0..5 = -x, +x, -y, +y, -z, +z), cell q = u + 8 v in the in-face
// coordinates of the halo loader of march_brick, holding the known value or
// +inf.  A march pass reads its neighbours' faces and the faces of the bricks
// it marched are rebuilt after the pass (which >= 0: work list `which`), so
// a pass sees the state of the previous one whatever the order of its
// marches.  which < 0: every brick.
template <typename real>
__global__ void k_faces_build(Geom g, const real *__restrict__ T, const uint8_t *__restrict__ tag,
                              const Control *ctrl, const int *list, int which, real *faces)
{
    const long long nb = which < 0 ? g.nbricks : (long long)ctrl->n_list[which];
    const long long n = nb * (kFaces * 64);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const long long bi = e / (kFaces * 64);
        const int r = (int)(e - bi * (kFaces * 64));
        const long long b = which < 0 ? bi : (long long)list[bi];
        const int f = r >> 6, q = r & 63, u = q & 7, v = q >> 3;
        const int axis = f >> 1;
        const int edge = (f & 1) ? kB - 1 : 0;
        const int cx = axis == 0 ? edge : u;
        const int cy = axis == 1 ? edge : (axis == 0 ? u : v);
        const int cz = axis == 2 ? edge : v;
        const long long ci = b * kB3 + cx + kB * cy + kB * kB * cz;
        faces[b * (kFaces * 64) + r] = is_known(tag[ci]) ? T[ci] : inf_v<real>();
    }
}

template <typename real>
void faces_build(const Geom &g, const DeviceState &s, int which, cudaStream_t st)
{
    const int nb = grid_for(g.nbricks * (kFaces * 64), 256, 152 * 32);
    k_faces_build<real><<<nb, 256, 0, st>>>(g, (const real *)s.T, s.tag, s.ctrl,
                                            which < 0 ? nullptr : s.list[which], which, (real *)s.faces);
}

// Trace: restart, phase and list length of a march launch.
__global__ void k_trace(const Control *c, int which, int phase, int *out)
{
    out[0] = c->done ? -1 : c->restart;
    out[1] = phase;
    out[2] = c->done ? 0 : (int)c->n_list[which];
}

__global__ void k_trace_seed(const Control *c, int *out)
{
    out[0] = c->done ? -1 : c->restart;
    out[1] = 0;
    out[2] = c->done ? 0 : (int)c->q_tail;
}

__global__ void k_reset_list(Control *c, int which)
{
    if (c->done)
        return;
    c->n_list[which] = 0u;
    c->work[which] = 0u;
}

// Calls f with the speed-field, tape and unequal-cell flags as compile-time
// constants (std::true_type / std::false_type), one kernel instantiation per
// combination.
template <typename Fn>
void with_flags(bool het, bool tape, bool aniso, Fn &&f)
{
    using Y = std::true_type;
    using N = std::false_type;
    auto third = [&](auto H, auto P) {
        if (aniso)
            f(H, P, Y{});
        else
            f(H, P, N{});
    };
    if (het) {
        if (tape)
            third(Y{}, Y{});
        else
            third(Y{}, N{});
    } else if (tape) {
        third(N{}, Y{});
    } else {
        third(N{}, N{});
    }
}

template <typename real>
cudaError_t restart_impl(const Geom &g, const DeviceState &s, const SolveParams &p,
                         cudaStream_t st, cudaEvent_t *ev, int *trace)
{
    const int rb = grid_for(g.nbricks, 256, 4096);
    const bool het = s.spd != nullptr, tape = s.tape != nullptr;
    const double sct = p.spd_term;
    k_reduce<real><<<rb, 256, 0, st>>>(g, (const real *)s.bmin, s.inmin, s.dirty, s.ctrl);
    k_control<<<1, 1, 0, st>>>(s.ctrl, p.width, p.stride, p.max_restarts);
    if (one_launch_schedule(p.schedule)) {
        k_seed<real><<<rb, 256, 0, st>>>(g, (const real *)s.bmin, s.inmin, s.ctrl, s.queued, s.queue);
        if (trace)
            k_trace_seed<<<1, 1, 0, st>>>(s.ctrl, trace);
        if (ev)
            cudaEventRecord(ev[0], st);
        with_flags(het, tape, p.aniso != 0, [&](auto H, auto P, auto A) {
            constexpr bool h = decltype(H)::value, t = decltype(P)::value, an = decltype(A)::value;
            const size_t sm = march_smem<real, t>();
            if (p.schedule == kScheduleContinuous)
                k_march_continuous<real, h, t, an><<<s.march_ctas, kMarchWarps * 32, sm, st>>>(g, s, p, sct);
            else
                k_march_persistent<real, h, t, an><<<s.march_ctas, kMarchWarps * 32, sm, st>>>(g, s, p, sct);
        });
        if (ev)
            cudaEventRecord(ev[1], st);
        return cudaGetLastError();
    }
    for (int pass = 0; pass <= p.passes; ++pass) {
        const int which = pass == 0 ? 0 : 1;
        if (pass >= 2)
            k_reset_list<<<1, 1, 0, st>>>(s.ctrl, 1);
        k_select<real><<<rb, 256, 0, st>>>(g, (const real *)s.bmin, s.dirty, s.fresh, s.inbox,
                                           s.ctrl, s.list[which], which);
        if (trace)
            k_trace<<<1, 1, 0, st>>>(s.ctrl, which, pass, trace + 3 * pass);
        if (ev)
            cudaEventRecord(ev[2 * pass], st);
        with_flags(het, tape, p.aniso != 0, [&](auto H, auto P, auto A) {
            k_march<real, decltype(H)::value, 1, decltype(P)::value, decltype(A)::value>
                <<<s.march_ctas, kMarchWarps * 32, march_smem<real, decltype(P)::value>(), st>>>(g, s, p, sct,
                                                                                                  which);
        });
        if (s.faces)
            faces_build<real>(g, s, which, st);
        if (ev)
            cudaEventRecord(ev[2 * pass + 1], st);
    }
    return cudaGetLastError();
}

template <typename real>
cudaError_t front_init_impl(const Geom &g, const DeviceState &s, const SolveParams &p,
                            cudaStream_t st)
{
    const long long need = (g.nbricks + kMarchWarps - 1) / kMarchWarps;
    const int nb = (int)(need < s.march_ctas ? need : s.march_ctas);
    with_flags(s.spd != nullptr, s.tape != nullptr, p.aniso != 0, [&](auto H, auto P, auto A) {
        k_march<real, decltype(H)::value, 0, decltype(P)::value, decltype(A)::value>
            <<<nb, kMarchWarps * 32, march_smem<real, decltype(P)::value>(), st>>>(g, s, p, p.spd_term, 0);
    });
    if (s.faces)
        faces_build<real>(g, s, -1, st);
    return cudaGetLastError();
}

// Shared-memory attributes of every march kernel; returns the resident CTAs
// per SM of the march kernels with or without the tape (the smallest over
// the kernels a solve may launch).
template <typename real>
int configure_march(bool tape)
{
    const auto attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
    int n = 1 << 20;
    for (int f = 0; f < 8; ++f)
        with_flags((f & 1) != 0, (f & 2) != 0, (f & 4) != 0, [&](auto H, auto P, auto A) {
            constexpr bool hh = decltype(H)::value, tt = decltype(P)::value, an = decltype(A)::value;
            const int sm = (int)march_smem<real, tt>();
            cudaFuncSetAttribute(k_march<real, hh, 1, tt, an>, attr, sm);
            cudaFuncSetAttribute(k_march<real, hh, 0, tt, an>, attr, sm);
            cudaFuncSetAttribute(k_march_persistent<real, hh, tt, an>, attr, sm);
            cudaFuncSetAttribute(k_march_continuous<real, hh, tt, an>, attr, sm);
            if (tt != tape)
                return;
            int k = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k, k_march_continuous<real, hh, tt, an>,
                                                          kMarchWarps * 32, sm);
            n = k < n ? k : n;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k, k_march<real, hh, 1, tt, an>, kMarchWarps * 32,
                                                          sm);
            n = k < n ? k : n;
        });
    return n > 0 && n < (1 << 20) ? n : 1;
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

cudaError_t launch_init_sources(int dtype, const Geom &g, const DeviceState &s,
                                const long long *src_ijk, long long n_src, cudaStream_t st)
{
    const int nb = grid_for(g.nbricks, 1, 152 * 16);
    if (dtype == 1) {
        k_init_sources<double><<<nb, 256, 0, st>>>(g, (double *)s.T, s.tag);
        if (n_src > 0)
            k_set_sources<double><<<grid_for(n_src, 256, 1024), 256, 0, st>>>(g, src_ijk, n_src,
                                                                             (double *)s.T, s.tag);
    } else {
        k_init_sources<float><<<nb, 256, 0, st>>>(g, (float *)s.T, s.tag);
        if (n_src > 0)
            k_set_sources<float><<<grid_for(n_src, 256, 1024), 256, 0, st>>>(g, src_ijk, n_src,
                                                                            (float *)s.T, s.tag);
    }
    return cudaGetLastError();
}

cudaError_t launch_init_reinit(int dtype, const Geom &g, const DeviceState &s,
                               const SolveParams &p, const void *phi0, cudaStream_t st, int zlo,
                               int zhi)
{
    const int nb = grid_for(g.nbricks, 1, 152 * 16);
    const long long layer = (long long)g.nx * g.ny;
    if (dtype == 1)
        k_init_reinit<double><<<nb, 256, 0, st>>>(g, p.h, p.hy, p.hz, (const double *)phi0 + zlo * layer,
                                                  (double *)s.T, s.tag, zlo, zhi);
    else
        k_init_reinit<float><<<nb, 256, 0, st>>>(g, p.h, p.hy, p.hz, (const float *)phi0 + zlo * layer,
                                                 (float *)s.T, s.tag, zlo, zhi);
    return cudaGetLastError();
}

cudaError_t launch_load_speed(int dtype, const Geom &g, const DeviceState &s, double h,
                              double hmin, const void *speed, double speed_const, cudaStream_t st)
{
    const int nb = grid_for(g.nbricks, 1, 152 * 8);
    if (dtype == 1)
        k_load_speed<double><<<nb, kThreads, 0, st>>>(g, h, hmin, (const double *)speed, speed_const,
                                                      (double *)s.spd, (double *)s.bdelta, s.ctrl);
    else
        k_load_speed<float><<<nb, kThreads, 0, st>>>(g, h, hmin, (const float *)speed, speed_const,
                                                     (float *)s.spd, (float *)s.bdelta, s.ctrl);
    return cudaGetLastError();
}

cudaError_t launch_front_init(int dtype, const Geom &g, const DeviceState &s,
                              const SolveParams &p, cudaStream_t st)
{
    return dtype == 1 ? front_init_impl<double>(g, s, p, st) : front_init_impl<float>(g, s, p, st);
}

cudaError_t launch_restart(int dtype, const Geom &g, const DeviceState &s, const SolveParams &p,
                           cudaStream_t st, cudaEvent_t *ev, int *trace)
{
    return dtype == 1 ? restart_impl<double>(g, s, p, st, ev, trace)
                      : restart_impl<float>(g, s, p, st, ev, trace);
}

cudaError_t launch_reset_control(const DeviceState &s, cudaStream_t st, unsigned long long wait_ns,
                                 int hold)
{
    k_reset_control<<<1, 1, 0, st>>>(s.ctrl, wait_ns, hold);
    return cudaGetLastError();
}

cudaError_t launch_output(int dtype, const Geom &g, const DeviceState &s, void *T_out,
                          uint8_t *tags_out, cudaStream_t st)
{
    const int nb = grid_for(g.nbricks, 1, 152 * 16);
    if (dtype == 1)
        k_output<double><<<nb, kInitThreads, 0, st>>>(g, (const double *)s.T, s.tag, (double *)T_out,
                                                      tags_out);
    else
        k_output<float><<<nb, kInitThreads, 0, st>>>(g, (const float *)s.T, s.tag, (float *)T_out,
                                                     tags_out);
    return cudaGetLastError();
}

cudaError_t launch_layer_export(int dtype, const Geom &g, const DeviceState &s, int z0, int nl,
                                void *out, cudaStream_t st)
{
    const int nb = grid_for((long long)g.nx * g.ny * nl, 256, 152 * 32);
    if (dtype == 1)
        k_layer_export<double><<<nb, 256, 0, st>>>(g, (const double *)s.T, s.tag, z0, nl, (double *)out);
    else
        k_layer_export<float><<<nb, 256, 0, st>>>(g, (const float *)s.T, s.tag, z0, nl, (float *)out);
    return cudaGetLastError();
}

cudaError_t launch_layer_integrate(int dtype, const Geom &g, const DeviceState &s, int z0, int nl,
                                   const void *in, unsigned *count, cudaStream_t st)
{
    const int nb = grid_for((long long)g.nx * g.ny * nl, 256, 152 * 32);
    if (dtype == 1)
        k_layer_integrate<double><<<nb, 256, 0, st>>>(g, (double *)s.T, s.tag, (double *)s.bmin, z0, nl,
                                                      (const double *)in, count);
    else
        k_layer_integrate<float><<<nb, 256, 0, st>>>(g, (float *)s.T, s.tag, (float *)s.bmin, z0, nl,
                                                     (const float *)in, count);
    return cudaGetLastError();
}

// One march of Algorithm 12 to a given bound: every brick with a BAND cell
// at or below it marches, and bricks whose halo changed march again, until
// none is left (the persistent queue).
cudaError_t launch_march_to(int dtype, const Geom &g, const DeviceState &s, const SolveParams &p,
                            double b0, double b1, cudaStream_t st)
{
    k_set_bound<<<1, 1, 0, st>>>(s.ctrl, b0, b1);
    const int rb = grid_for(g.nbricks, 256, 4096);
    const bool het = s.spd != nullptr, tape = s.tape != nullptr;
    if (dtype == 1) {
        k_seed<double><<<rb, 256, 0, st>>>(g, (const double *)s.bmin, s.inmin, s.ctrl, s.queued, s.queue);
        with_flags(het, tape, p.aniso != 0, [&](auto H, auto P, auto A) {
            k_march_persistent<double, decltype(H)::value, decltype(P)::value, decltype(A)::value>
                <<<s.march_ctas, kMarchWarps * 32, march_smem<double, decltype(P)::value>(), st>>>(g, s, p,
                                                                                                   p.spd_term);
        });
    } else {
        k_seed<float><<<rb, 256, 0, st>>>(g, (const float *)s.bmin, s.inmin, s.ctrl, s.queued, s.queue);
        with_flags(het, tape, p.aniso != 0, [&](auto H, auto P, auto A) {
            k_march_persistent<float, decltype(H)::value, decltype(P)::value, decltype(A)::value>
                <<<s.march_ctas, kMarchWarps * 32, march_smem<float, decltype(P)::value>(), st>>>(g, s, p,
                                                                                                  p.spd_term);
        });
    }
    return cudaGetLastError();
}

// The per-side BAND minima of the grid (Algorithm 16's local heap tops) into
// the control block (minbits).
cudaError_t launch_minima(int dtype, const Geom &g, const DeviceState &s, cudaStream_t st)
{
    k_set_bound<<<1, 1, 0, st>>>(s.ctrl, 0.0, 0.0);
    const int rb = grid_for(g.nbricks, 256, 4096);
    if (dtype == 1)
        k_reduce<double><<<rb, 256, 0, st>>>(g, (const double *)s.bmin, s.inmin, s.dirty, s.ctrl);
    else
        k_reduce<float><<<rb, 256, 0, st>>>(g, (const float *)s.bmin, s.inmin, s.dirty, s.ctrl);
    return cudaGetLastError();
}

cudaError_t launch_select(int dtype, const Geom &g, const DeviceState &s, int which,
                          cudaStream_t st)
{
    const int rb = grid_for(g.nbricks, 256, 4096);
    if (dtype == 1)
        k_select<double><<<rb, 256, 0, st>>>(g, (const double *)s.bmin, s.dirty, s.fresh, s.inbox,
                                             s.ctrl, s.list[which], which);
    else
        k_select<float><<<rb, 256, 0, st>>>(g, (const float *)s.bmin, s.dirty, s.fresh, s.inbox,
                                            s.ctrl, s.list[which], which);
    return cudaGetLastError();
}

cudaError_t launch_reset_list(const DeviceState &s, int which, cudaStream_t st)
{
    k_reset_list<<<1, 1, 0, st>>>(s.ctrl, which);
    return cudaGetLastError();
}

cudaError_t launch_batch_init(int dtype, const BatchGrid *grids, const int *bgrid,
                              long long nbricks, const DeviceState &s, cudaStream_t st)
{
    const int nb = grid_for(nbricks * kB3, 256, 152 * 32);
    if (dtype == 1)
        k_batch_init<double><<<nb, 256, 0, st>>>(grids, bgrid, nbricks, (double *)s.T, s.tag);
    else
        k_batch_init<float><<<nb, 256, 0, st>>>(grids, bgrid, nbricks, (float *)s.T, s.tag);
    return cudaGetLastError();
}

cudaError_t launch_batch_sources(int dtype, const BatchGrid *grids, const long long *src,
                                 long long n_src, const DeviceState &s, cudaStream_t st)
{
    if (n_src <= 0)
        return cudaSuccess;
    const int nb = grid_for(n_src, 256, 1024);
    if (dtype == 1)
        k_batch_sources<double><<<nb, 256, 0, st>>>(grids, src, n_src, (double *)s.T, s.tag);
    else
        k_batch_sources<float><<<nb, 256, 0, st>>>(grids, src, n_src, (float *)s.T, s.tag);
    return cudaGetLastError();
}

cudaError_t launch_batch_speed(int dtype, const BatchGrid *grids, const int *bgrid,
                               long long nbricks, const DeviceState &s, cudaStream_t st)
{
    const int nb = grid_for(nbricks, 1, 152 * 8);
    if (dtype == 1)
        k_batch_speed<double><<<nb, kThreads, 0, st>>>(grids, bgrid, nbricks, (double *)s.spd,
                                                       (double *)s.bdelta, s.ctrl);
    else
        k_batch_speed<float><<<nb, kThreads, 0, st>>>(grids, bgrid, nbricks, (float *)s.spd,
                                                      (float *)s.bdelta, s.ctrl);
    return cudaGetLastError();
}

cudaError_t launch_batch_output(int dtype, const BatchGrid *grids, const int *bgrid,
                                long long nbricks, const DeviceState &s, cudaStream_t st)
{
    const int nb = grid_for(nbricks * kB3, 256, 152 * 32);
    if (dtype == 1)
        k_batch_output<double><<<nb, 256, 0, st>>>(grids, bgrid, nbricks, (const double *)s.T, s.tag);
    else
        k_batch_output<float><<<nb, 256, 0, st>>>(grids, bgrid, nbricks, (const float *)s.T, s.tag);
    return cudaGetLastError();
}

cudaError_t launch_faces_build(int dtype, const Geom &g, const DeviceState &s, cudaStream_t st)
{
    if (dtype == 1)
        faces_build<double>(g, s, -1, st);
    else
        faces_build<float>(g, s, -1, st);
    return cudaGetLastError();
}

int march_blocks_per_sm(int dtype, bool tape)
{
    return dtype == 1 ? configure_march<double>(tape) : configure_march<float>(tape);
}

}  // namespace fmmgb
