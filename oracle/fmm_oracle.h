/*
 * fmm_oracle.h -- ORACLE: plain sequential fp64 narrow band fast marching.
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, obviously correct CPU
 * statement of what the CUDA library computes.  Only the test suite, the smoke
 * check of the build entry point and the CPU-baseline leg of the benchmark may
 * load it.  It shares no code, header, table or helper with the CUDA library.
 *
 * Grid convention (Sec. 2.1): psi lives at the centres of cells of size
 * dx * dy * dz, uniform in each direction; h3 = {dx, dy, dz} (all > 0) gives
 * the h_i = 1/dx, 1/dy, 1/dz of Algorithm 11.  Arrays are nx*ny*nz doubles,
 * x fastest: idx = (k*ny + j)*nx + i.  Neighbours outside the grid are simply absent
 * (Sec. 4.1: no boundary conditions, stencils never leave the array).
 *
 * Tags are the augmented status tags of Sec. 4.2.  In a single-process run
 * only FAR, BAND_NEW, KNOWN_FIX and KNOWN_NEW occur.
 *
 * All functions return 0 on success and a negative value on bad arguments or
 * allocation failure.
 */
#ifndef FMM_ORACLE_H
#define FMM_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    ORC_FAR = 0,
    ORC_BAND_NEW = 1,
    ORC_BAND_OLD = 2,
    ORC_KNOWN_FIX = 3,
    ORC_KNOWN_NEW = 4,
    ORC_KNOWN_OLD = 5
};

/* Algorithm 8 for point sources: psi <- +inf, G <- FAR everywhere, then each
 * listed source cell (i,j,k triples, 3*nsrc int64) gets psi = 0, KNOWN_FIX. */
int oracle_init_sources(int64_t nx, int64_t ny, int64_t nz,
                        const int64_t *src_ijk, int64_t nsrc,
                        double *T, uint8_t *G);

/* Algorithm 8 for a signed level set phi0: cells that have a 6-neighbour of
 * the opposite sign (sign(0) = +1) are the cells adjacent to the interface.
 * They get psi = sign * (sum over crossing axes of d_a^-2)^(-1/2), where d_a
 * is the smaller linear-interpolation crossing distance on axis a (a fraction
 * of that axis's cell size), and KNOWN_FIX.  Every other cell gets +inf and
 * FAR (Algorithm 8 assigns +inf). */
int oracle_init_reinit(int64_t nx, int64_t ny, int64_t nz, const double h3[3],
                       const double *phi0, double *T, uint8_t *G);

/* Algorithm 9 followed by Algorithm 12 with bound_band(+-1) = width (the
 * sequential reference of Sec. 5.2).  T and G come from an init call and are
 * updated in place.  speed == NULL means a constant speed speed_const.  A
 * cell with F = 0 is an obstacle (test case 6 of Sec. 5.1): its term
 * F^-2 = +inf gives no finite root, so it stays FAR with psi = +inf.
 * Optional outputs (NULL to skip):
 *   order[n]   : cell indices in acceptance (heap pop) order; *n_order = count
 *   tape[n]    : for each cell, the upwind set of the root that gave its final
 *                value: 2 bits per axis (x bits 0-1, y 2-3, z 4-5),
 *                0 = axis unused, 1 = minus neighbour, 2 = plus neighbour. */
int oracle_march(int64_t nx, int64_t ny, int64_t nz, const double h3[3],
                 const double *speed, double speed_const, double width,
                 double *T, uint8_t *G,
                 int64_t *order, int64_t *n_order, uint8_t *tape);

/* Algorithm 11 on one cell, given the values of its 6 neighbours in the order
 * -x,+x,-y,+y,-z,+z.  nb_known[q] != 0 marks a neighbour that exists and is
 * KNOWN.  Tc is the cell's current |psi| (the upwind filter of Algorithm 11);
 * F is the speed at the cell.  Returns psi_temp (+inf if no causal root). */
double oracle_local_solve(const double nb[6], const uint8_t nb_known[6],
                          double Tc, const double h3[3], double F);

/* The higher-order fast marching that Sec. 6 names as future work, with the
 * restarted-band march unchanged: oracle_march with accuracy 2 replaces the
 * first-order difference on an upwind axis by the second-order one-sided
 * difference (3 t - 4 psi1 + psi2) / (2 h) wherever the cell psi2 two steps
 * away on that side is KNOWN and |psi2| <= |psi1|; elsewhere, and everywhere
 * for accuracy 1, the axis is first order as in Eq. (2)-(3).  No tape: the
 * adjoint and tangent below linearise the first-order scheme only.  Returns
 * -1 for an accuracy other than 1 or 2. */
int oracle_march_ho(int64_t nx, int64_t ny, int64_t nz, const double h3[3],
                    const double *speed, double speed_const, double width,
                    double *T, uint8_t *G,
                    int64_t *order, int64_t *n_order, int accuracy);

/* oracle_local_solve with the second-order difference of oracle_march_ho:
 * nb2[q] / nb2_known[q] are the cells two steps away in the same six
 * directions. */
double oracle_local_solve_ho(const double nb[6], const uint8_t nb_known[6],
                             const double nb2[6], const uint8_t nb2_known[6],
                             double Tc, const double h3[3], double F);

/* Gauss-Seidel fast sweeping (Zhao 2005, cited in Sec. 1) with the textbook
 * sorted Godunov update of Eq. (2) over all six neighbours (the per-axis
 * minima sorted together with their cell sizes).  A holds |psi|:
 * cells with fixed[idx] != 0 keep their value, the rest start at +inf.
 * Sweeps in the 8 alternating orders until a full round changes nothing or
 * max_rounds rounds are done; *rounds_out receives the count. */
int oracle_fast_sweep(int64_t nx, int64_t ny, int64_t nz, const double h3[3],
                      const double *speed, double speed_const,
                      double *A, const uint8_t *fixed,
                      int64_t max_rounds, int64_t *rounds_out);

/* Reverse-mode derivative of L(T) with respect to the slowness s = 1/F, with
 * the upwind sets of the tape held fixed.  At an accepted non-FIX cell p the
 * discrete equation sum_{i in U(p)} ((T_p - T_i)/h_i)^2 = s_p^2 (h_i the cell
 * size along the axis of neighbour i) gives
 *   dT_p/ds_p = s_p / D_p,  dT_p/dT_i = (T_p - T_i)/(h_i^2 D_p),
 *   D_p = sum_{i in U(p)} (T_p - T_i)/h_i^2,
 * applied in reverse acceptance order.  FIX cells absorb lambda.  Inputs are
 * the outputs of oracle_march (|T| is used, so both sides work).
 * lambda (nullable) receives the total adjoint dL/dT_p. */
int oracle_adjoint(int64_t nx, int64_t ny, int64_t nz, const double h3[3],
                   const double *speed, double speed_const,
                   const double *T, const uint8_t *G, const uint8_t *tape,
                   const int64_t *order, int64_t n_order,
                   const double *dLdT, double *dLds, double *lambda);

/* Forward-mode tangent dT = J v for a slowness perturbation v, with the same
 * linearisation as oracle_adjoint, applied in acceptance order. */
int oracle_tangent(int64_t nx, int64_t ny, int64_t nz, const double h3[3],
                   const double *speed, double speed_const,
                   const double *T, const uint8_t *G, const uint8_t *tape,
                   const int64_t *order, int64_t n_order,
                   const double *v, double *dT);

#ifdef __cplusplus
}
#endif
#endif /* FMM_ORACLE_H */
