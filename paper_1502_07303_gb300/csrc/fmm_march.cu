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
//   March_Narrow_Band_Parallel (Alg. 12)    -> k_march<mode 1> on a work list
//   Collect/Exchange/Integrate (Alg. 13-15) -> write-back to HBM plus per-face
//                                               "fresh" bit masks and a dirty
//                                               flag on the neighbour brick; the
//                                               neighbour's next staging reads
//                                               the new values
//   second march of Alg. 16                 -> k_march<mode 1> on the bricks
//                                               made dirty by the first march
//
// Inside a brick the heap of Algorithm 12 is replaced by a bucketed,
// label-correcting march: each round accepts every BAND cell whose |psi| is
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

#include <cfloat>
#include <cmath>
#include <math_constants.h>

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

// ---------------------------------------------------------------------------
// Algorithm 11 (Solve_Quadratic_Parallel) on a staged tile.
//
// kv holds the value of every KNOWN/FIX cell of the brick and its halo and
// +inf elsewhere, so "G in KNOWN and |psi_n| < |psi_cell|" is "kv_n < Tc".
// The per-axis choice and the loop that drops the largest psi_i follow the
// algorithm; the root of the smallest causal set wins.  set_out receives
// the upwind set of the returned root (2 bits per axis: 1 = minus, 2 = plus).
// ---------------------------------------------------------------------------

// Double precision: the coefficients a, b, c of Algorithm 11 written with
// round-to-nearest intrinsics so that no multiply-add is fused.
__device__ __forceinline__ double solve_cell(const double *kv, int ti, double Tc, double finv2,
                                             double w, uint8_t &set_out)
{
    const int off[3] = {1, kTile, kTile * kTile};
    double psi[3], wa[3];
    int nd = 0;
    unsigned cur = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double vm = kv[ti - off[a]], vp = kv[ti + off[a]];
        int d = 0;
        if (vm < Tc)
            d = -1;
        if (vp < Tc && (d == 0 || vp < vm))
            d = 1;
        psi[a] = d == 0 ? 0.0 : (d < 0 ? vm : vp);
        wa[a] = d == 0 ? 0.0 : w;
        if (d != 0) {
            ++nd;
            cur |= (d < 0 ? 1u : 2u) << (2 * a);
        }
    }
    double best = inf_v<double>();
    unsigned best_set = 0;
#pragma unroll 1
    while (nd != 0) {
        const double qa = __dadd_rn(__dadd_rn(wa[0], wa[1]), wa[2]);
        const double sb = __dadd_rn(__dadd_rn(__dmul_rn(wa[0], psi[0]), __dmul_rn(wa[1], psi[1])),
                                    __dmul_rn(wa[2], psi[2]));
        const double qb = -2.0 * sb;
        const double sc =
            __dadd_rn(__dadd_rn(__dmul_rn(__dmul_rn(wa[0], psi[0]), psi[0]),
                                __dmul_rn(__dmul_rn(wa[1], psi[1]), psi[1])),
                      __dmul_rn(__dmul_rn(wa[2], psi[2]), psi[2]));
        const double qc = __dsub_rn(sc, finv2);
        const double disc = __dsub_rn(__dmul_rn(qb, qb), __dmul_rn(4.0 * qa, qc));
        if (disc >= 0.0) {
            const double t = __ddiv_rn(__dadd_rn(-qb, __dsqrt_rn(disc)), 2.0 * qa);
            if (psi[0] < t && psi[1] < t && psi[2] < t && t < best) {
                best = t;
                best_set = cur;
            }
        }
        // drop the axis with the largest psi still in the stencil (ties: the
        // higher axis index)
        int j = -1;
#pragma unroll
        for (int a = 0; a < 3; ++a)
            if (wa[a] != 0.0 && (j < 0 || psi[a] >= (j == 0 ? psi[0] : (j == 1 ? psi[1] : psi[2]))))
                j = a;
#pragma unroll
        for (int a = 0; a < 3; ++a)
            if (a == j) {
                psi[a] = 0.0;
                wa[a] = 0.0;
            }
        cur &= ~(3u << (2 * j));
        --nd;
    }
    set_out = (uint8_t)best_set;
    return best;
}

// Single precision: the same algorithm with the unknown shifted by the
// smallest upwind value (t = m + u, delta_i = psi_i - m, sum (u - delta_i)^2
// = (h/F)^2), which keeps the quadratic well conditioned when psi >> h.
__device__ __forceinline__ float solve_cell(const float *kv, int ti, float Tc, float q,
                                            double /*w*/, uint8_t &set_out)
{
    const int off[3] = {1, kTile, kTile * kTile};
    float psi[3];
    bool act[3];
    int nd = 0;
    unsigned cur = 0;
    float m = inf_v<float>();
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float vm = kv[ti - off[a]], vp = kv[ti + off[a]];
        int d = 0;
        if (vm < Tc)
            d = -1;
        if (vp < Tc && (d == 0 || vp < vm))
            d = 1;
        act[a] = d != 0;
        psi[a] = d == 0 ? 0.f : (d < 0 ? vm : vp);
        if (d != 0) {
            ++nd;
            cur |= (d < 0 ? 1u : 2u) << (2 * a);
            m = fminf(m, psi[a]);
        }
    }
    float del[3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
        del[a] = act[a] ? psi[a] - m : 0.f;
    float best = inf_v<float>();
    unsigned best_set = 0;
#pragma unroll 1
    while (nd != 0) {
        float S = 0.f, Q = 0.f;
#pragma unroll
        for (int a = 0; a < 3; ++a)
            if (act[a]) {
                S += del[a];
                Q += del[a] * del[a];
            }
        const float k = (float)nd;
        const float disc = S * S - k * (Q - q);
        if (disc >= 0.f) {
            const float u = (S + sqrtf(disc)) / k;
            bool causal = true;
#pragma unroll
            for (int a = 0; a < 3; ++a)
                causal = causal && (!act[a] || del[a] < u);
            const float t = m + u;
            if (causal && t < best) {
                best = t;
                best_set = cur;
            }
        }
        int j = -1;
        float dj = 0.f;
#pragma unroll
        for (int a = 0; a < 3; ++a)
            if (act[a] && (j < 0 || del[a] >= dj)) {
                j = a;
                dj = del[a];
            }
#pragma unroll
        for (int a = 0; a < 3; ++a)
            if (a == j)
                act[a] = false;
        cur &= ~(3u << (2 * j));
        --nd;
    }
    set_out = (uint8_t)best_set;
    return best;
}

template <typename real>
__device__ __forceinline__ real warp_min(real v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// ---------------------------------------------------------------------------
// Algorithm 8: interface initialisation, written directly in brick layout.
// ---------------------------------------------------------------------------

template <typename real>
__global__ void k_init_sources(Geom g, real *T, uint8_t *tag)
{
    const long long n = g.nbricks * kB3;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        int bx, by, bz;
        brick_coords(g, e >> 9, bx, by, bz);
        const int c = (int)(e & 511);
        const int i = bx * kB + (c & 7), j = by * kB + ((c >> 3) & 7), k = bz * kB + (c >> 6);
        const bool out = i >= g.nx || j >= g.ny || k >= g.nz;
        T[e] = inf_v<real>();
        tag[e] = out ? (uint8_t)(TG_OUT | ST_FAR) : (uint8_t)ST_FAR;
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

template <typename real>
__global__ void k_init_reinit(Geom g, double h, const real *__restrict__ phi, real *T,
                              uint8_t *tag)
{
    const long long n = g.nbricks * kB3;
    const long long sx = 1, sy = g.nx, sz = (long long)g.nx * g.ny;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        int bx, by, bz;
        brick_coords(g, e >> 9, bx, by, bz);
        const int c = (int)(e & 511);
        const int i = bx * kB + (c & 7), j = by * kB + ((c >> 3) & 7), k = bz * kB + (c >> 6);
        if (i >= g.nx || j >= g.ny || k >= g.nz) {
            T[e] = inf_v<real>();
            tag[e] = TG_OUT | ST_FAR;
            continue;
        }
        const long long p = (long long)k * sz + (long long)j * sy + i;
        const real fc = phi[p];
        const bool pos = fc >= (real)0;
        real d[3];
        bool any = false;
        const int co[3] = {i, j, k};
        const int ext[3] = {g.nx, g.ny, g.nz};
        const long long st[3] = {sx, sy, sz};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            d[a] = inf_v<real>();
#pragma unroll
            for (int dir = -1; dir <= 1; dir += 2) {
                const int q = co[a] + dir;
                if (q < 0 || q >= ext[a])
                    continue;
                const real fq = phi[p + dir * st[a]];
                if ((fq >= (real)0) == pos)
                    continue;
                const real dist = crossing(fc, fq, h);
                if (dist < d[a])
                    d[a] = dist;
                any = true;
            }
        }
        if (!any) {
            T[e] = inf_v<real>();
            tag[e] = pos ? (uint8_t)ST_FAR : (uint8_t)(ST_FAR | TG_NEG);
            continue;
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
        T[e] = zero ? (real)0 : inv_sqrt_exact(inv);
        tag[e] = pos ? (uint8_t)ST_FIX : (uint8_t)(ST_FIX | TG_NEG);
    }
}

// Speed field to brick layout.  Double precision keeps 1/F^2 (the F^-2 term of
// Algorithm 11); single precision keeps (h/F)^2 for the shifted solve.  Each
// brick also records its bucket width h * min(1/F) / sqrt(3).
__device__ __forceinline__ double speed_term(double F, double h) { return __ddiv_rn(1.0, __dmul_rn(F, F)); }
__device__ __forceinline__ float speed_term(float F, double h)
{
    const float hf = (float)h;
    return (hf * hf) / (F * F);
}

template <typename real>
__global__ void __launch_bounds__(kThreads) k_load_speed(Geom g, double h, const real *__restrict__ speed,
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
        if (!(F > (real)0) || !(F < inf_v<real>()))
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
            bdelta[b] = (real)(h / (1.7320508075688772 * (double)m));
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// The brick march.  kMode 0: Algorithm 9 (relax every non-FIX cell next to a
// FIX cell once, accept nothing) over all bricks.  kMode 1: Algorithm 12 up to
// the restart bound over the bricks of work list `which`.
// ---------------------------------------------------------------------------

template <typename real>
struct MarchShared {
    real kv[kTile3];
    real red[2][kThreads / 32];
    unsigned int facebits[kFaces][2];
    unsigned int outbits[kFaces][2];
    uint8_t acc[kB3];
};

__device__ __forceinline__ bool face_bit(const unsigned (*bits)[2], int f, int q)
{
    return (bits[f][q >> 5] >> (q & 31)) & 1u;
}

template <typename real, bool kHetero, int kMode>
__global__ void __launch_bounds__(kThreads, 2)
    k_march(Geom g, DeviceState s, SolveParams p, double spd_const_term, int which)
{
    __shared__ MarchShared<real> sh;
    Control *ctrl = s.ctrl;
    if (kMode == 1 && ctrl->done)
        return;
    const long long n = (kMode == 0) ? g.nbricks : (long long)ctrl->n_list[which];
    real *T = (real *)s.T;
    uint8_t *tag = s.tag;
    const real *spd = (const real *)s.spd;
    const real *bdelta = (const real *)s.bdelta;
    real *bmin = (real *)s.bmin;
    const int t = threadIdx.x;
    const int x = t & 7, y = (t >> 3) & 7, z = t >> 6;
    const int ti = (x + 1) + kTile * (y + 1) + kTile * kTile * (z + 1);
    const real INF = inf_v<real>();
    const real bound0 = (real)ctrl->bound[0], bound1 = (real)ctrl->bound[1];

    for (long long it = blockIdx.x; it < n; it += gridDim.x) {
        const long long b = (kMode == 0) ? it : (long long)s.list[which][it];
        int bx, by, bz;
        brick_coords(g, b, bx, by, bz);
        const long long base = b * kB3;

        // ---- stage the brick (owned: plain loads) -------------------------
        real tv = T[base + t];
        uint8_t tg = tag[base + t];
        const real sp = kHetero ? spd[base + t] : (real)spd_const_term;
        uint8_t tp = s.tape ? s.tape[base + t] : (uint8_t)0;
        const real kv0 = is_known(tg) ? tv : INF;
        sh.kv[ti] = kv0;
        if (t < 2 * kFaces)
            (&sh.outbits[0][0])[t] = 0u;
        if (kMode == 1 && t == 0) {
            // consume the pending-change flag and masks before reading the
            // halo: a change flagged after this point marks the brick again
            atomicExch(&s.dirty[b], 0u);
            __threadfence();
#pragma unroll
            for (int f = 0; f < kFaces; ++f) {
                const unsigned long long m = atomicExch(&s.fresh[b * kFaces + f], 0ull);
                sh.facebits[f][0] = (unsigned)m;
                sh.facebits[f][1] = (unsigned)(m >> 32);
            }
            __threadfence();
        }
        __syncthreads();

        // ---- halo: the neighbour bricks' boundary layers (read-only) -------
        if (t < kFaces * 64) {
            const int f = t >> 6, q = t & 63, u = q & 7, v = q >> 3;
            const int axis = f >> 1, dir = (f & 1) ? 1 : -1;
            const int nbx = bx + (axis == 0 ? dir : 0);
            const int nby = by + (axis == 1 ? dir : 0);
            const int nbz = bz + (axis == 2 ? dir : 0);
            real val = INF;
            if (nbx >= 0 && nbx < g.nbx && nby >= 0 && nby < g.nby && nbz >= 0 && nbz < g.nbz) {
                const int edge = dir < 0 ? kB - 1 : 0;
                const int cx = axis == 0 ? edge : u;
                const int cy = axis == 1 ? edge : (axis == 0 ? u : v);
                const int cz = axis == 2 ? edge : v;
                const long long nb = ((long long)nbz * g.nby + nby) * g.nbx + nbx;
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
            sh.kv[hx + kTile * hy + kTile * kTile * hz] = val;
        }
        __syncthreads();

        const bool frozen = ((tg & ST_MASK) == ST_FIX) || (tg & TG_OUT);
        const bool neg = (tg & TG_NEG) != 0;
        bool relax = false;
        if (!frozen) {
            if (kMode == 0) {
                relax = sh.kv[ti - 1] < tv || sh.kv[ti + 1] < tv || sh.kv[ti - kTile] < tv ||
                        sh.kv[ti + kTile] < tv || sh.kv[ti - kTile * kTile] < tv ||
                        sh.kv[ti + kTile * kTile] < tv;
            } else {
                const unsigned(*fb)[2] = sh.facebits;
                if (x == 0 && face_bit(fb, 0, y + 8 * z) && sh.kv[ti - 1] < tv) relax = true;
                if (x == 7 && face_bit(fb, 1, y + 8 * z) && sh.kv[ti + 1] < tv) relax = true;
                if (y == 0 && face_bit(fb, 2, x + 8 * z) && sh.kv[ti - kTile] < tv) relax = true;
                if (y == 7 && face_bit(fb, 3, x + 8 * z) && sh.kv[ti + kTile] < tv) relax = true;
                if (z == 0 && face_bit(fb, 4, x + 8 * y) && sh.kv[ti - kTile * kTile] < tv) relax = true;
                if (z == 7 && face_bit(fb, 5, x + 8 * y) && sh.kv[ti + kTile * kTile] < tv) relax = true;
            }
        }

        const real delta = (real)p.bucket * bdelta[b];
        int rounds = 0;
        long long n_acc = 0;
        real m0 = INF, m1 = INF;
        for (;;) {
            // Algorithm 10/11: re-solve next to the newly accepted cells
            real cand = INF;
            uint8_t cset = 0;
            if (relax)
                cand = solve_cell(sh.kv, ti, tv, sp, p.w, cset);
            __syncthreads();
            if (cand < tv) {
                tv = cand;
                tg = (uint8_t)((tg & ~ST_MASK) | ST_BAND);
                sh.kv[ti] = INF;
                tp = cset;
            }
            // minimum of the BAND cells of each side (the heap tops)
            const bool band = (tg & ST_MASK) == ST_BAND;
            real b0 = warp_min<real>(band && neg ? tv : INF);
            real b1 = warp_min<real>(band && !neg ? tv : INF);
            if ((t & 31) == 0) {
                sh.red[0][t >> 5] = b0;
                sh.red[1][t >> 5] = b1;
            }
            __syncthreads();
            m0 = sh.red[0][0];
            m1 = sh.red[1][0];
#pragma unroll
            for (int w = 1; w < kThreads / 32; ++w) {
                m0 = fmin(m0, sh.red[0][w]);
                m1 = fmin(m1, sh.red[1][w]);
            }
            if (kMode == 0)
                break;
            // accept the lowest bucket up to the restart bound
            const real lim = neg ? fmin(m0 + delta, bound0) : fmin(m1 + delta, bound1);
            const bool acc = band && tv <= lim;
            if (acc) {
                tg = (uint8_t)((tg & ~ST_MASK) | ST_KNOWN);
                sh.kv[ti] = tv;
            }
            sh.acc[t] = acc;
            const int na = __syncthreads_count(acc);
            if (na == 0)
                break;
            n_acc += na;
            if (++rounds > p.max_rounds) {
                if (t == 0)
                    atomicOr(&ctrl->error, ERR_ROUNDS);
                break;
            }
            relax = false;
            if (!frozen) {
                if (x > 0 && sh.acc[t - 1] && sh.kv[ti - 1] < tv) relax = true;
                if (x < 7 && sh.acc[t + 1] && sh.kv[ti + 1] < tv) relax = true;
                if (y > 0 && sh.acc[t - 8] && sh.kv[ti - kTile] < tv) relax = true;
                if (y < 7 && sh.acc[t + 8] && sh.kv[ti + kTile] < tv) relax = true;
                if (z > 0 && sh.acc[t - 64] && sh.kv[ti - kTile * kTile] < tv) relax = true;
                if (z < 7 && sh.acc[t + 64] && sh.kv[ti + kTile * kTile] < tv) relax = true;
            }
        }

        // ---- write back, front minima, overlap change notification --------
        T[base + t] = tv;
        tag[base + t] = tg;
        if (s.tape)
            s.tape[base + t] = tp;
        if (t == 0) {
            bmin[2 * b] = m0;
            bmin[2 * b + 1] = m1;
        }
        if (kMode == 1) {
            const real kvf = is_known(tg) ? tv : INF;
            if (kvf < kv0) {
                unsigned(*ob)[2] = sh.outbits;
                if (x == 0) atomicOr(&ob[0][(y + 8 * z) >> 5], 1u << ((y + 8 * z) & 31));
                if (x == 7) atomicOr(&ob[1][(y + 8 * z) >> 5], 1u << ((y + 8 * z) & 31));
                if (y == 0) atomicOr(&ob[2][(x + 8 * z) >> 5], 1u << ((x + 8 * z) & 31));
                if (y == 7) atomicOr(&ob[3][(x + 8 * z) >> 5], 1u << ((x + 8 * z) & 31));
                if (z == 0) atomicOr(&ob[4][(x + 8 * y) >> 5], 1u << ((x + 8 * y) & 31));
                if (z == 7) atomicOr(&ob[5][(x + 8 * y) >> 5], 1u << ((x + 8 * y) & 31));
            }
            __threadfence();
            __syncthreads();
            if (t < kFaces) {
                const int f = t;
                const unsigned long long m =
                    (unsigned long long)sh.outbits[f][0] | ((unsigned long long)sh.outbits[f][1] << 32);
                const int axis = f >> 1, dir = (f & 1) ? 1 : -1;
                const int nbx = bx + (axis == 0 ? dir : 0);
                const int nby = by + (axis == 1 ? dir : 0);
                const int nbz = bz + (axis == 2 ? dir : 0);
                if (m && nbx >= 0 && nbx < g.nbx && nby >= 0 && nby < g.nby && nbz >= 0 &&
                    nbz < g.nbz) {
                    const long long nb = ((long long)nbz * g.nby + nby) * g.nbx + nbx;
                    atomicOr(&s.fresh[nb * kFaces + (f ^ 1)], m);
                    atomicExch(&s.dirty[nb], 1u);
                    atomicAdd(&ctrl->exchanges, (unsigned long long)__popcll(m));
                }
            }
            if (t == 0) {
                atomicAdd(&ctrl->marches, 1ull);
                atomicAdd(&ctrl->rounds, (unsigned long long)rounds);
                atomicAdd(&ctrl->accepted, (unsigned long long)n_acc);
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Algorithm 16 bookkeeping: global minima of the front, exit test, bound.
// ---------------------------------------------------------------------------

template <typename real>
__global__ void k_reduce(Geom g, const real *__restrict__ bmin, const unsigned *__restrict__ dirty,
                         Control *ctrl)
{
    if (ctrl->done)
        return;
    __shared__ double r0[8], r1[8];
    __shared__ unsigned rc[8];
    double m0 = CUDART_INF, m1 = CUDART_INF;
    unsigned cnt = 0;
    for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b < g.nbricks;
         b += (long long)gridDim.x * blockDim.x) {
        m0 = fmin(m0, (double)bmin[2 * b]);
        m1 = fmin(m1, (double)bmin[2 * b + 1]);
        cnt += dirty[b] != 0u;
    }
    m0 = warp_min<double>(m0);
    m1 = warp_min<double>(m1);
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
    const unsigned long long INF_BITS = 0x7ff0000000000000ull;
    double mv0 = fmin(__longlong_as_double((long long)c->minbits[0]), width);
    double mv1 = fmin(__longlong_as_double((long long)c->minbits[1]), width);
    c->restart += 1;
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
}

// Work lists: list 0 = bricks with a BAND cell at or below the bound or with
// pending overlap changes (first march); list 1 = bricks with pending changes
// (second march, after the exchange).
template <typename real>
__global__ void k_select(Geom g, const real *__restrict__ bmin, const unsigned *__restrict__ dirty,
                         Control *ctrl, int *list, int which)
{
    if (ctrl->done)
        return;
    const double bd0 = ctrl->bound[0], bd1 = ctrl->bound[1];
    const int lane = threadIdx.x & 31;
    for (long long b0 = blockIdx.x * (long long)blockDim.x; b0 < g.nbricks;
         b0 += (long long)gridDim.x * blockDim.x) {
        const long long b = b0 + threadIdx.x;
        bool sel = false;
        if (b < g.nbricks) {
            sel = dirty[b] != 0u;
            if (which == 0)
                sel = sel || (double)bmin[2 * b] <= bd0 || (double)bmin[2 * b + 1] <= bd1;
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

__global__ void k_reset_control(Control *c)
{
    const unsigned long long INF_BITS = 0x7ff0000000000000ull;
    c->minbits[0] = INF_BITS;
    c->minbits[1] = INF_BITS;
    c->marches = c->rounds = c->exchanges = c->accepted = 0ull;
    c->bound[0] = c->bound[1] = 0.0;
    c->dirty_count = 0u;
    c->n_list[0] = c->n_list[1] = 0u;
    c->done = 0;
    c->error = 0;
    c->restart = 0;
}

// Brick layout -> the caller's x-fastest arrays (signed psi, public tags).
template <typename real>
__global__ void k_output(Geom g, const real *__restrict__ T, const uint8_t *__restrict__ tag,
                         real *T_out, uint8_t *tags_out)
{
    const long long n = (long long)g.nx * g.ny * g.nz;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(p % g.nx);
        const long long r = p / g.nx;
        const int j = (int)(r % g.ny), k = (int)(r / g.ny);
        const long long b = ((long long)(k >> 3) * g.nby + (j >> 3)) * g.nbx + (i >> 3);
        const long long e = b * kB3 + (i & 7) + 8 * (j & 7) + 64 * (k & 7);
        const real v = T[e];
        const uint8_t tg = tag[e];
        const uint8_t st = tg & ST_MASK;
        real out = v;
        if (st == ST_FAR)
            out = inf_v<real>();
        else if (tg & TG_NEG)
            out = -v;
        T_out[p] = out;
        if (tags_out)
            tags_out[p] = st;
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

template <typename real>
cudaError_t restart_impl(const Geom &g, const DeviceState &s, const SolveParams &p,
                         cudaStream_t st, cudaEvent_t *ev4)
{
    const int rb = grid_for(g.nbricks, 256, 4096);
    const bool het = s.spd != nullptr;
    const double sct = p.spd_term;
    k_reduce<real><<<rb, 256, 0, st>>>(g, (const real *)s.bmin, s.dirty, s.ctrl);
    k_control<<<1, 1, 0, st>>>(s.ctrl, p.width, p.stride, p.max_restarts);
    for (int which = 0; which < 2; ++which) {
        k_select<real><<<rb, 256, 0, st>>>(g, (const real *)s.bmin, s.dirty, s.ctrl,
                                           s.list[which], which);
        if (ev4)
            cudaEventRecord(ev4[2 * which], st);
        if (het)
            k_march<real, true, 1><<<s.march_ctas, kThreads, 0, st>>>(g, s, p, sct, which);
        else
            k_march<real, false, 1><<<s.march_ctas, kThreads, 0, st>>>(g, s, p, sct, which);
        if (ev4)
            cudaEventRecord(ev4[2 * which + 1], st);
    }
    return cudaGetLastError();
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

cudaError_t launch_init_sources(int dtype, const Geom &g, const DeviceState &s,
                                const long long *src_ijk, long long n_src, cudaStream_t st)
{
    const int nb = grid_for(g.nbricks * kB3, 256, 152 * 32);
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
                               const SolveParams &p, const void *phi0, cudaStream_t st)
{
    const int nb = grid_for(g.nbricks * kB3, 256, 152 * 32);
    if (dtype == 1)
        k_init_reinit<double><<<nb, 256, 0, st>>>(g, p.h, (const double *)phi0, (double *)s.T, s.tag);
    else
        k_init_reinit<float><<<nb, 256, 0, st>>>(g, p.h, (const float *)phi0, (float *)s.T, s.tag);
    return cudaGetLastError();
}

cudaError_t launch_load_speed(int dtype, const Geom &g, const DeviceState &s, double h,
                              const void *speed, double speed_const, cudaStream_t st)
{
    const int nb = grid_for(g.nbricks, 1, 152 * 8);
    if (dtype == 1)
        k_load_speed<double><<<nb, kThreads, 0, st>>>(g, h, (const double *)speed, speed_const,
                                                      (double *)s.spd, (double *)s.bdelta, s.ctrl);
    else
        k_load_speed<float><<<nb, kThreads, 0, st>>>(g, h, (const float *)speed, speed_const,
                                                     (float *)s.spd, (float *)s.bdelta, s.ctrl);
    return cudaGetLastError();
}

cudaError_t launch_front_init(int dtype, const Geom &g, const DeviceState &s,
                              const SolveParams &p, cudaStream_t st)
{
    const bool het = s.spd != nullptr;
    const int nb = (int)(g.nbricks < s.march_ctas ? g.nbricks : s.march_ctas);
    if (dtype == 1) {
        if (het)
            k_march<double, true, 0><<<nb, kThreads, 0, st>>>(g, s, p, p.spd_term, 0);
        else
            k_march<double, false, 0><<<nb, kThreads, 0, st>>>(g, s, p, p.spd_term, 0);
    } else {
        if (het)
            k_march<float, true, 0><<<nb, kThreads, 0, st>>>(g, s, p, p.spd_term, 0);
        else
            k_march<float, false, 0><<<nb, kThreads, 0, st>>>(g, s, p, p.spd_term, 0);
    }
    return cudaGetLastError();
}

cudaError_t launch_restart(int dtype, const Geom &g, const DeviceState &s, const SolveParams &p,
                           cudaStream_t st, cudaEvent_t *ev4)
{
    return dtype == 1 ? restart_impl<double>(g, s, p, st, ev4) : restart_impl<float>(g, s, p, st, ev4);
}

cudaError_t launch_reset_control(const DeviceState &s, cudaStream_t st)
{
    k_reset_control<<<1, 1, 0, st>>>(s.ctrl);
    return cudaGetLastError();
}

cudaError_t launch_output(int dtype, const Geom &g, const DeviceState &s, void *T_out,
                          uint8_t *tags_out, cudaStream_t st)
{
    const long long n = (long long)g.nx * g.ny * g.nz;
    const int nb = grid_for(n, 256, 152 * 32);
    if (dtype == 1)
        k_output<double><<<nb, 256, 0, st>>>(g, (const double *)s.T, s.tag, (double *)T_out, tags_out);
    else
        k_output<float><<<nb, 256, 0, st>>>(g, (const float *)s.T, s.tag, (float *)T_out, tags_out);
    return cudaGetLastError();
}

int march_blocks_per_sm(int dtype)
{
    int n = 0;
    if (dtype == 1)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_march<double, true, 1>, kThreads, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_march<float, true, 1>, kThreads, 0);
    return n > 0 ? n : 1;
}

}  // namespace fmmgb
