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
// lambda_p = g_p + sum_q mu_q (T_q - T_p).  One warp processes one 8^3 brick
// in rounds (the cells that became ready in a round are computed together);
// downwind neighbours in other bricks are read from their published mu.  A
// brick that finished boundary cells marks the bricks holding their upwind
// neighbours dirty, and the dirty bricks run again (the select kernel of the
// forward path builds the list) until no brick is dirty.  The order of the
// sums is fixed, so the result is deterministic.
#include "fmm_internal.h"

#include <cmath>

namespace fmmgb {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int kAdjWarps = 4;

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

template <typename real>
__global__ void k_adj_init(Geom g, const uint8_t *__restrict__ tag, real *mu, real *dlds)
{
    const long long n = g.nbricks * kB3;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        int bx, by, bz;
        brick_xyz(g, e >> 9, bx, by, bz);
        const int c = (int)(e & 511);
        const int i = bx * kB + (c & 7), j = by * kB + ((c >> 3) & 7), k = bz * kB + (c >> 6);
        mu[e] = accepted(tag[e]) ? nan_v<real>() : (real)0;
        if (i < g.nx && j < g.ny && k < g.nz)
            dlds[((long long)k * g.ny + j) * g.nx + i] = (real)0;
    }
}

template <typename real>
struct AdjTile {
    real T[kTile3];      // |psi| of the brick and its face halo
    real mu[kTile3];     // published mu (NaN = not done) of brick and halo
    uint8_t tp[kTile3];  // tape of brick and halo
    uint8_t tg[kB3];     // tags of the brick
};

__device__ __forceinline__ int tile_of(int c)
{
    return 111 + (c & 7) + kTile * ((c >> 3) & 7) + kTile * kTile * (c >> 6);
}

// Tape code of axis a of cell tp: 0 none, 1 minus neighbour, 2 plus.
__device__ __forceinline__ int tape_axis(uint8_t tp, int a) { return (tp >> (2 * a)) & 3; }

template <typename real>
__device__ __forceinline__ bool is_nan(real v) { return v != v; }

template <typename real, bool kHetero, int kMode>
__global__ void __launch_bounds__(kAdjWarps * 32)
    k_adj_march(Geom g, DeviceState s, const real *__restrict__ dLdT, real *dlds, real *mu_g,
                double h, double spd_const_term, int which)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    AdjTile<real> &W = reinterpret_cast<AdjTile<real> *>(smem_raw)[warp];
    Control *ctrl = s.ctrl;
    const long long n = (kMode == 0) ? g.nbricks : (long long)ctrl->n_list[which];
    const int *work_list = which ? s.list[1] : s.list[0];
    const real *T = (const real *)s.T;
    const real *spd = (const real *)s.spd;
    const int off[3] = {1, kTile, kTile * kTile};
    for (long long it = (long long)blockIdx.x * kAdjWarps + warp; it < n;
         it += (long long)gridDim.x * kAdjWarps) {
        const long long b = (kMode == 0) ? it : (long long)work_list[it];
        int bx, by, bz;
        brick_xyz(g, b, bx, by, bz);
        const long long base = b * kB3;
        // ---- stage T, mu, tape of the brick ------------------------------
#pragma unroll 4
        for (int k = 0; k < 16; ++k) {
            const int c = lane + 32 * k;
            const int ti = tile_of(c);
            W.T[ti] = T[base + c];
            W.mu[ti] = mu_g[base + c];
            W.tp[ti] = s.tape[base + c];
            W.tg[c] = s.tag[base + c];
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
                tpv = s.tape[ci];
                mv = __ldcg(mu_g + ci);
                if (!accepted(s.tag[ci]))
                    tpv = 0;   // only accepted cells have upwind sets
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
        // interior cells that are not accepted have no upwind set either
#pragma unroll 4
        for (int k = 0; k < 16; ++k) {
            const int c = lane + 32 * k;
            if (!accepted(W.tg[c]))
                W.tp[tile_of(c)] = 0;
        }
        __syncwarp();

        // ---- rounds: cells whose downwind neighbours have all published ---
        unsigned face_done = 0;   // bit f: a done cell has an upwind cell across face f
        for (int round = 0; round < 4096; ++round) {
            int progressed = 0;
#pragma unroll 2
            for (int k = 0; k < 16; ++k) {
                const int c = lane + 32 * k;
                const int ti = tile_of(c);
                const real mup = W.mu[ti];
                bool ready = false;
                real lam = (real)0, dsum = (real)0;
                if (is_nan(mup)) {
                    ready = true;
                    const real Tp = W.T[ti];
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        // neighbours on axis a: q = p - e_a (its upwind code 2
                        // points at p) and q = p + e_a (code 1 points at p);
                        // halo entries of missing bricks and cells that were
                        // not accepted carry tape 0
                        const int qm = ti - off[a], qp = ti + off[a];
                        if (tape_axis(W.tp[qm], a) == 2) {
                            const real m = W.mu[qm];
                            if (is_nan(m))
                                ready = false;
                            else
                                lam += m * (W.T[qm] - Tp);
                        }
                        if (tape_axis(W.tp[qp], a) == 1) {
                            const real m = W.mu[qp];
                            if (is_nan(m))
                                ready = false;
                            else
                                lam += m * (W.T[qp] - Tp);
                        }
                        const int code = tape_axis(W.tp[ti], a);
                        if (code)
                            dsum += Tp - W.T[code == 1 ? qm : qp];
                    }
                }
                // the 32 cells of this step read before any of them publishes
                __syncwarp();
                if (ready) {
                    const int cx = c & 7, cy = (c >> 3) & 7, cz = c >> 6;
                    const int i = bx * kB + cx, j = by * kB + cy, kk = bz * kB + cz;
                    const long long nat = ((long long)kk * g.ny + j) * g.nx + i;
                    lam += dLdT[nat];
                    const real m = dsum > (real)0 ? lam / dsum : (real)0;
                    W.mu[ti] = m;
                    const real q = kHetero ? spd[base + c] : (real)spd_const_term;
                    const real sh2 = sqrt(q) * (real)h;   // s_p h^2 with q = (h/F)^2
                    dlds[nat] = m * sh2;
                    const uint8_t tpc = W.tp[ti];
                    if (cx == 0 && tape_axis(tpc, 0) == 1) face_done |= 1u;
                    if (cx == 7 && tape_axis(tpc, 0) == 2) face_done |= 2u;
                    if (cy == 0 && tape_axis(tpc, 1) == 1) face_done |= 4u;
                    if (cy == 7 && tape_axis(tpc, 1) == 2) face_done |= 8u;
                    if (cz == 0 && tape_axis(tpc, 2) == 1) face_done |= 16u;
                    if (cz == 7 && tape_axis(tpc, 2) == 2) face_done |= 32u;
                    progressed = 1;
                }
                __syncwarp();
            }
            if (!__any_sync(FULL, progressed))
                break;
        }
        // ---- publish mu, wake the bricks that hold upwind neighbours ------
#pragma unroll 4
        for (int k = 0; k < 16; ++k) {
            const int c = lane + 32 * k;
            mu_g[base + c] = W.mu[tile_of(c)];
        }
        face_done = __reduce_or_sync(FULL, face_done);
        if (lane < kFaces && ((face_done >> lane) & 1u)) {
            const int f = lane, axis = f >> 1, dir = (f & 1) ? 1 : -1;
            const int nbx = bx + (axis == 0 ? dir : 0);
            const int nby = by + (axis == 1 ? dir : 0);
            const int nbz = bz + (axis == 2 ? dir : 0);
            if (nbx >= 0 && nbx < g.nbx && nby >= 0 && nby < g.nby && nbz >= 0 && nbz < g.nbz)
                s.dirty[((long long)nbz * g.nby + nby) * g.nbx + nbx] = 1u;
        }
        __syncwarp();
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
cudaError_t adj_launch(const Geom &g, const DeviceState &s, const AdjointArgs &a, int mode,
                       int which, cudaStream_t st)
{
    const size_t sm = adj_smem<real>();
    const int ctas = s.march_ctas;
    const bool het = s.spd != nullptr;
    if (mode == 0) {
        if (het)
            k_adj_march<real, true, 0><<<ctas, kAdjWarps * 32, sm, st>>>(
                g, s, (const real *)a.dLdT, (real *)a.dlds, (real *)a.mu, a.h, a.spd_term, which);
        else
            k_adj_march<real, false, 0><<<ctas, kAdjWarps * 32, sm, st>>>(
                g, s, (const real *)a.dLdT, (real *)a.dlds, (real *)a.mu, a.h, a.spd_term, which);
    } else {
        if (het)
            k_adj_march<real, true, 1><<<ctas, kAdjWarps * 32, sm, st>>>(
                g, s, (const real *)a.dLdT, (real *)a.dlds, (real *)a.mu, a.h, a.spd_term, which);
        else
            k_adj_march<real, false, 1><<<ctas, kAdjWarps * 32, sm, st>>>(
                g, s, (const real *)a.dLdT, (real *)a.dlds, (real *)a.mu, a.h, a.spd_term, which);
    }
    return cudaGetLastError();
}

template <typename real>
void adj_configure()
{
    const int sm = (int)adj_smem<real>();
    cudaFuncSetAttribute(k_adj_march<real, true, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_adj_march<real, false, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_adj_march<real, true, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_adj_march<real, false, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
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
    if (dtype == 1) {
        adj_configure<double>();
        k_adj_init<double><<<nb, 256, 0, st>>>(g, s.tag, (double *)a.mu, (double *)a.dlds);
    } else {
        adj_configure<float>();
        k_adj_init<float><<<nb, 256, 0, st>>>(g, s.tag, (float *)a.mu, (float *)a.dlds);
    }
    return cudaGetLastError();
}

cudaError_t launch_adjoint_march(int dtype, const Geom &g, const DeviceState &s,
                                 const AdjointArgs &a, int mode, int which, cudaStream_t st)
{
    return dtype == 1 ? adj_launch<double>(g, s, a, mode, which, st)
                      : adj_launch<float>(g, s, a, mode, which, st);
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
