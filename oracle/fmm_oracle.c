/*
 * fmm_oracle.c -- ORACLE: plain sequential fp64 narrow band fast marching.
 *
 * TEST INFRASTRUCTURE ONLY (see fmm_oracle.h).  Nothing on the product path
 * may call into this file; it shares no code with the CUDA library.
 *
 * What it computes.  The paper's sequential reference of Sec. 5.2: the
 * parallel algorithm reduced to Algorithm 8 (interface initialisation),
 * Algorithm 9 (heap initialisation) and one instance of Algorithm 12 (march)
 * with bound_band = width_band, using Algorithm 10 (neighbour update) and
 * Algorithm 11 (quadratic solve) for the first-order Godunov upwind scheme of
 * Eq. (2)-(3).  The two-sided heap of Sec. 3 is kept as two ordinary binary
 * heaps, one per side; that behaves the same as the paper's single array with
 * negative indices.  Heap ties (equal |psi|) pop the smaller linear index
 * first; the paper is silent on ties.
 *
 * oracle_march_ho adds the higher-order fast marching of Sec. 6 (future work
 * there): the same march with second-order one-sided differences on the axes
 * where the next cell beyond the upwind neighbour is known and monotone.
 *
 * Build: plain C11, -ffp-contract=off so that no multiply-add is fused and
 * x86-64 and aarch64 produce the same bits.
 */
#include "fmm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* the cell sizes (dx, dy, dz) of Sec. 2.1 must be positive */
static int spacing_ok(const double h3[3])
{
    return h3 && h3[0] > 0 && h3[1] > 0 && h3[2] > 0;
}

#define OR_INF INFINITY

static int is_known(uint8_t g)
{
    return g == ORC_KNOWN_FIX || g == ORC_KNOWN_NEW || g == ORC_KNOWN_OLD;
}

/* ------------------------------------------------------------------------ */
/* Grid helpers                                                              */
/* ------------------------------------------------------------------------ */

typedef struct {
    int64_t nx, ny, nz, n;
    int64_t ext[3];
    int64_t stride[3];
} grid_t;

static int grid_make(grid_t *g, int64_t nx, int64_t ny, int64_t nz)
{
    if (nx <= 0 || ny <= 0 || nz <= 0)
        return -1;
    g->nx = nx;
    g->ny = ny;
    g->nz = nz;
    g->n = nx * ny * nz;
    g->ext[0] = nx;
    g->ext[1] = ny;
    g->ext[2] = nz;
    g->stride[0] = 1;
    g->stride[1] = nx;
    g->stride[2] = nx * ny;
    return 0;
}

static void grid_coord(const grid_t *g, int64_t idx, int64_t c[3])
{
    c[0] = idx % g->nx;
    c[1] = (idx / g->nx) % g->ny;
    c[2] = idx / (g->nx * g->ny);
}

/* Index of the neighbour of idx along axis a in direction d (-1 or +1), or
 * -1 when it lies outside the grid. */
static int64_t grid_nb(const grid_t *g, int64_t idx, const int64_t c[3],
                       int a, int d)
{
    int64_t q = c[a] + d;
    if (q < 0 || q >= g->ext[a])
        return -1;
    return idx + d * g->stride[a];
}

static double speed_at(const double *speed, double speed_const, int64_t idx)
{
    return speed ? speed[idx] : speed_const;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 8: interface initialisation                                      */
/* ------------------------------------------------------------------------ */

int oracle_init_sources(int64_t nx, int64_t ny, int64_t nz,
                        const int64_t *src_ijk, int64_t nsrc,
                        double *T, uint8_t *G)
{
    grid_t g;
    if (grid_make(&g, nx, ny, nz) || !T || !G || nsrc < 0 ||
        (nsrc > 0 && !src_ijk))
        return -1;
    for (int64_t p = 0; p < g.n; ++p) {
        T[p] = OR_INF;       /* psi <- +inf */
        G[p] = ORC_FAR;      /* G <- FAR    */
    }
    for (int64_t s = 0; s < nsrc; ++s) {
        int64_t i = src_ijk[3 * s], j = src_ijk[3 * s + 1],
                k = src_ijk[3 * s + 2];
        if (i < 0 || i >= nx || j < 0 || j >= ny || k < 0 || k >= nz)
            return -2;
        int64_t p = (k * ny + j) * nx + i;
        T[p] = 0.0;
        G[p] = ORC_KNOWN_FIX;
    }
    return 0;
}

int oracle_init_reinit(int64_t nx, int64_t ny, int64_t nz, const double h3[3],
                       const double *phi0, double *T, uint8_t *G)
{
    grid_t g;
    if (grid_make(&g, nx, ny, nz) || !phi0 || !T || !G || !spacing_ok(h3))
        return -1;
    for (int64_t p = 0; p < g.n; ++p) {
        int64_t c[3];
        grid_coord(&g, p, c);
        double fc = phi0[p];
        int sc = (fc >= 0.0) ? 1 : -1;
        int any = 0;
        double d_axis[3] = {OR_INF, OR_INF, OR_INF};
        for (int a = 0; a < 3; ++a) {
            for (int d = -1; d <= 1; d += 2) {
                int64_t q = grid_nb(&g, p, c, a, d);
                if (q < 0)
                    continue;
                double fq = phi0[q];
                int sq = (fq >= 0.0) ? 1 : -1;
                if (sq == sc)
                    continue;
                /* the interface crosses the segment p-q at fraction theta
                 * of the way from p (linear interpolation of phi0) */
                double theta = fc / (fc - fq);
                double dist = theta * h3[a];
                if (dist < d_axis[a])
                    d_axis[a] = dist;
                any = 1;
            }
        }
        if (!any) {
            T[p] = OR_INF;
            G[p] = ORC_FAR;
            continue;
        }
        double inv = 0.0;
        int zero = 0;
        for (int a = 0; a < 3; ++a) {
            if (d_axis[a] == OR_INF)
                continue;
            if (d_axis[a] == 0.0)
                zero = 1;
            else
                inv = inv + 1.0 / (d_axis[a] * d_axis[a]);
        }
        double mag = zero ? 0.0 : 1.0 / sqrt(inv);
        T[p] = (sc > 0) ? mag : -mag;
        G[p] = ORC_KNOWN_FIX;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Indexed binary min-heap keyed on |psi| (textbook, cited in Sec. 2.2)       */
/* ------------------------------------------------------------------------ */

typedef struct {
    int32_t *a;
    int64_t size, cap;
} heap_t;

typedef struct {
    grid_t g;
    double h3[3];       /* dx, dy, dz */
    const double *speed;
    double speed_const;
    double *T;
    uint8_t *G;
    uint8_t *tape;
    int32_t *pos;       /* position of each cell in its side's heap, or -1 */
    int8_t *side;       /* side of the heap holding the cell (-1/+1), or 0 */
    heap_t heap[2];     /* [0]: side -1, [1]: side +1 */
    int64_t *order;
    int64_t n_order;
    int accuracy;       /* 1: Eq. (2)-(3); 2: second-order upwind differences */
} march_t;

static int heap_less(const march_t *m, int32_t a, int32_t b)
{
    double ta = fabs(m->T[a]), tb = fabs(m->T[b]);
    return ta < tb || (ta == tb && a < b);
}

static void heap_set(march_t *m, heap_t *hp, int64_t i, int32_t cell)
{
    hp->a[i] = cell;
    m->pos[cell] = (int32_t)i;
}

static void up_heap(march_t *m, heap_t *hp, int64_t i)
{
    int32_t cell = hp->a[i];
    while (i > 0) {
        int64_t parent = (i - 1) / 2;
        if (!heap_less(m, cell, hp->a[parent]))
            break;
        heap_set(m, hp, i, hp->a[parent]);
        i = parent;
    }
    heap_set(m, hp, i, cell);
}

static void down_heap(march_t *m, heap_t *hp, int64_t i)
{
    int32_t cell = hp->a[i];
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, best = i;
        int32_t best_cell = cell;
        if (l < hp->size && heap_less(m, hp->a[l], best_cell)) {
            best = l;
            best_cell = hp->a[l];
        }
        if (r < hp->size && heap_less(m, hp->a[r], best_cell)) {
            best = r;
            best_cell = hp->a[r];
        }
        if (best == i)
            break;
        heap_set(m, hp, i, best_cell);
        i = best;
    }
    heap_set(m, hp, i, cell);
}

static int insert_heap(march_t *m, heap_t *hp, int32_t cell)
{
    if (hp->size == hp->cap) {
        int64_t ncap = hp->cap ? 2 * hp->cap : 1024;
        int32_t *na = (int32_t *)realloc(hp->a, (size_t)ncap * sizeof(int32_t));
        if (!na)
            return -3;
        hp->a = na;
        hp->cap = ncap;
    }
    hp->size += 1;
    heap_set(m, hp, hp->size - 1, cell);
    up_heap(m, hp, hp->size - 1);
    return 0;
}

static int32_t remove_min(march_t *m, heap_t *hp)
{
    int32_t top = hp->a[0];
    m->pos[top] = -1;
    hp->size -= 1;
    if (hp->size > 0) {
        hp->a[0] = hp->a[hp->size];
        m->pos[hp->a[0]] = 0;
        down_heap(m, hp, 0);
    }
    return top;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 11: Solve_Quadratic_Parallel                                    */
/* ------------------------------------------------------------------------ */

/* psi[a], hh[a] per axis as in Algorithm 11 (hh = 1/h or 0); dir[a] is the
 * chosen neighbour direction (-1, +1 or 0).  Returns psi_temp and the upwind
 * set of the root that produced it (2 bits per axis, see the header).
 *
 * The quadratic of Algorithm 11, sum_i h_i^2 (t - psi_i)^2 = F^-2, is solved
 * for the unknown shifted by the smallest upwind value m: t = m + u with
 * delta_i = psi_i - m, giving a = sum h_i^2, b = -2 sum h_i^2 delta_i and
 * c = sum h_i^2 delta_i^2 - F^-2.  It is the same equation; written in psi
 * itself, b^2 and 4ac are of order (psi/h)^2 while b^2 - 4ac is of order
 * (1/(hF))^2, so rounding would cost about 3 (psi F/h)^2 ulp in the
 * discriminant (1e-10 relative at 1024^3), far from the machine-accuracy
 * agreement of parallel and sequential solutions reported in Sec. 5.2.  The
 * causality test psi_i < t reads delta_i < u in the shifted unknown. */
static double quadratic_roots(double psi[3], double hh[3], const int dir[3],
                              double Finv2, uint8_t *set_out)
{
    uint8_t cur = 0;
    int nd = 0;
    double m = OR_INF;
    for (int a = 0; a < 3; ++a) {
        if (hh[a] != 0.0) {
            nd += 1;
            cur |= (uint8_t)((dir[a] < 0 ? 1 : 2) << (2 * a));
            if (psi[a] < m)
                m = psi[a];
        }
    }
    double psi_temp = OR_INF;
    uint8_t best_set = 0;
    while (nd != 0) {
        double d0 = hh[0] != 0.0 ? psi[0] - m : 0.0;
        double d1 = hh[1] != 0.0 ? psi[1] - m : 0.0;
        double d2 = hh[2] != 0.0 ? psi[2] - m : 0.0;
        double w0 = hh[0] * hh[0], w1 = hh[1] * hh[1], w2 = hh[2] * hh[2];
        double qa = (w0 + w1) + w2;
        double qb = -2.0 * (((w0 * d0) + (w1 * d1)) + (w2 * d2));
        double qc = ((((w0 * d0) * d0) + ((w1 * d1) * d1)) + ((w2 * d2) * d2)) - Finv2;
        double disc = qb * qb - (4.0 * qa) * qc;
        if (disc >= 0.0) {
            double u = (-qb + sqrt(disc)) / (2.0 * qa);
            if (d0 < u && d1 < u && d2 < u) {
                double t = m + u;
                if (t < psi_temp) {
                    psi_temp = t;
                    best_set = cur;
                }
            }
        }
        /* drop the axis with the largest psi among those still in the
         * stencil; on a tie the higher axis index goes first */
        int j = -1;
        for (int a = 0; a < 3; ++a)
            if (hh[a] != 0.0 && (j < 0 || psi[a] >= psi[j]))
                j = a;
        psi[j] = 0.0;
        hh[j] = 0.0;
        cur &= (uint8_t)~(3u << (2 * j));
        nd -= 1;
    }
    if (set_out)
        *set_out = best_set;
    return psi_temp;
}

/* Second-order upwind difference along one axis (the higher-order fast
 * marching that Sec. 6 names as future work; the scheme is the textbook
 * second-order FMM).  With psi1 the upwind neighbour and psi2 the next cell
 * beyond it in the same direction, the one-sided difference
 * (3 t - 4 psi1 + psi2) / (2 h) equals (3 / (2 h)) (t - (4 psi1 - psi2) / 3):
 * the axis enters Algorithm 11's quadratic unchanged, with
 * psi_i = (4 psi1 - psi2) / 3 and h_i = 3 / (2 h).  It is used only where
 * psi2 is KNOWN and not above psi1 (the values fall monotonically away from
 * the cell); otherwise the axis keeps the first-order difference. */
static void second_order_axis(double psi1, double psi2, int known2, double h,
                              double *psi, double *hh)
{
    if (known2 && psi2 <= psi1) {
        *psi = (4.0 * psi1 - psi2) / 3.0;
        *hh = 3.0 / (2.0 * h);
    }
}

static double solve_quadratic(const march_t *m, int64_t l, uint8_t *set_out)
{
    const grid_t *g = &m->g;
    int64_t c[3];
    grid_coord(g, l, c);
    double Tl = fabs(m->T[l]);
    double psi[3], hh[3];
    int dir[3];
    for (int a = 0; a < 3; ++a) {
        int d = 0;
        int64_t qm = grid_nb(g, l, c, a, -1);
        int64_t qp = grid_nb(g, l, c, a, +1);
        if (qm >= 0 && is_known(m->G[qm]) && fabs(m->T[qm]) < Tl)
            d = -1;
        if (qp >= 0 && is_known(m->G[qp]) && fabs(m->T[qp]) < Tl) {
            if (d == 0)
                d = 1;
            else if (fabs(m->T[qp]) < fabs(m->T[qm]))
                d = 1;
        }
        dir[a] = d;
        if (d != 0) {
            psi[a] = fabs(m->T[l + d * g->stride[a]]);
            hh[a] = 1.0 / m->h3[a];
            if (m->accuracy == 2) {
                int64_t c1[3] = {c[0], c[1], c[2]};
                c1[a] += d;
                int64_t q2 = grid_nb(g, l + d * g->stride[a], c1, a, d);
                if (q2 >= 0)
                    second_order_axis(psi[a], fabs(m->T[q2]), is_known(m->G[q2]),
                                      m->h3[a], &psi[a], &hh[a]);
            }
        } else {
            psi[a] = 0.0;
            hh[a] = 0.0;
        }
    }
    double F = speed_at(m->speed, m->speed_const, l);
    double Finv2 = 1.0 / (F * F);
    return quadratic_roots(psi, hh, dir, Finv2, set_out);
}

double oracle_local_solve(const double nb[6], const uint8_t nb_known[6],
                          double Tc, const double h3[3], double F)
{
    double psi[3], hh[3];
    int dir[3];
    double Tl = fabs(Tc);
    for (int a = 0; a < 3; ++a) {
        int d = 0;
        double vm = fabs(nb[2 * a]), vp = fabs(nb[2 * a + 1]);
        if (nb_known[2 * a] && vm < Tl)
            d = -1;
        if (nb_known[2 * a + 1] && vp < Tl) {
            if (d == 0)
                d = 1;
            else if (vp < vm)
                d = 1;
        }
        dir[a] = d;
        if (d != 0) {
            psi[a] = (d < 0) ? vm : vp;
            hh[a] = 1.0 / h3[a];
        } else {
            psi[a] = 0.0;
            hh[a] = 0.0;
        }
    }
    return quadratic_roots(psi, hh, dir, 1.0 / (F * F), NULL);
}

double oracle_local_solve_ho(const double nb[6], const uint8_t nb_known[6],
                             const double nb2[6], const uint8_t nb2_known[6],
                             double Tc, const double h3[3], double F)
{
    double psi[3], hh[3];
    int dir[3];
    double Tl = fabs(Tc);
    for (int a = 0; a < 3; ++a) {
        int d = 0;
        double vm = fabs(nb[2 * a]), vp = fabs(nb[2 * a + 1]);
        if (nb_known[2 * a] && vm < Tl)
            d = -1;
        if (nb_known[2 * a + 1] && vp < Tl) {
            if (d == 0)
                d = 1;
            else if (vp < vm)
                d = 1;
        }
        dir[a] = d;
        psi[a] = 0.0;
        hh[a] = 0.0;
        if (d != 0) {
            int q = 2 * a + (d < 0 ? 0 : 1);
            psi[a] = fabs(nb[q]);
            hh[a] = 1.0 / h3[a];
            second_order_axis(psi[a], fabs(nb2[q]), nb2_known[q] != 0, h3[a],
                              &psi[a], &hh[a]);
        }
    }
    return quadratic_roots(psi, hh, dir, 1.0 / (F * F), NULL);
}

/* ------------------------------------------------------------------------ */
/* Algorithm 10: Update_Neighbors_Parallel                                   */
/* ------------------------------------------------------------------------ */

static int update_neighbors(march_t *m, int64_t idx, int s)
{
    const grid_t *g = &m->g;
    int64_t c[3];
    grid_coord(g, idx, c);
    double Ti = fabs(m->T[idx]);
    heap_t *hp = &m->heap[s < 0 ? 0 : 1];
    for (int a = 0; a < 3; ++a) {
        for (int d = -1; d <= 1; d += 2) {
            int64_t l = grid_nb(g, idx, c, a, d);
            if (l < 0)
                continue;
            if (m->G[l] == ORC_KNOWN_FIX || !(fabs(m->T[l]) > Ti))
                continue;
            uint8_t set = 0;
            double t = solve_quadratic(m, l, &set);
            if (t < fabs(m->T[l])) {
                /* a cell queued on the other side would mean a non-FIX cell
                 * touches the opposite sign, which Algorithm 8 rules out
                 * (every sign change lies between two KNOWN_FIX cells) */
                if (m->pos[l] >= 0 && m->side[l] != s)
                    return -4;
                m->T[l] = (s < 0) ? -t : t;
                m->G[l] = ORC_BAND_NEW;
                if (m->tape)
                    m->tape[l] = set;
                if (m->pos[l] < 0) {
                    m->side[l] = (int8_t)s;
                    int rc = insert_heap(m, hp, (int32_t)l);
                    if (rc)
                        return rc;
                } else {
                    up_heap(m, hp, m->pos[l]);
                }
            }
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 9 + Algorithm 12 with bound = width                              */
/* ------------------------------------------------------------------------ */

static int march_run(int64_t nx, int64_t ny, int64_t nz, const double h3[3],
                     const double *speed, double speed_const, double width,
                     double *T, uint8_t *G,
                     int64_t *order, int64_t *n_order, uint8_t *tape, int accuracy)
{
    march_t m;
    memset(&m, 0, sizeof(m));
    if (grid_make(&m.g, nx, ny, nz) || !T || !G || !spacing_ok(h3))
        return -1;
    m.accuracy = accuracy;
    if (m.g.n >= (int64_t)2147483647)
        return -1;
    if (!speed && !(speed_const > 0))
        return -1;
    for (int a = 0; a < 3; ++a)
        m.h3[a] = h3[a];
    m.speed = speed;
    m.speed_const = speed_const;
    m.T = T;
    m.G = G;
    m.tape = tape;
    m.order = order;
    m.pos = (int32_t *)malloc((size_t)m.g.n * sizeof(int32_t));
    m.side = (int8_t *)calloc((size_t)m.g.n, sizeof(int8_t));
    if (!m.pos || !m.side) {
        free(m.pos);
        free(m.side);
        return -3;
    }
    for (int64_t p = 0; p < m.g.n; ++p)
        m.pos[p] = -1;
    if (tape)
        memset(tape, 0, (size_t)m.g.n);

    int rc = 0;
    /* Algorithm 9: every KNOWN_FIX cell updates its neighbours with side
     * s = sgn(psi), sgn(0) = +1 */
    for (int64_t p = 0; p < m.g.n && !rc; ++p) {
        if (G[p] != ORC_KNOWN_FIX)
            continue;
        int s = (T[p] >= 0.0) ? 1 : -1;
        rc = update_neighbors(&m, p, s);
    }
    /* Algorithm 12, bound_band(s) = width_band for both sides */
    for (int s = -1; s <= 1 && !rc; s += 2) {
        heap_t *hp = &m.heap[s < 0 ? 0 : 1];
        for (;;) {
            if (hp->size == 0)
                break;
            int32_t top = hp->a[0];               /* Locate_Min(s) */
            if (fabs(T[top]) > width)
                break;
            if (G[top] != ORC_KNOWN_OLD)
                G[top] = ORC_KNOWN_NEW;
            remove_min(&m, hp);
            if (order)
                order[m.n_order] = top;
            m.n_order += 1;
            rc = update_neighbors(&m, top, s);
            if (rc)
                break;
        }
    }
    if (n_order)
        *n_order = m.n_order;
    free(m.pos);
    free(m.side);
    free(m.heap[0].a);
    free(m.heap[1].a);
    return rc;
}

int oracle_march(int64_t nx, int64_t ny, int64_t nz, const double h3[3],
                 const double *speed, double speed_const, double width,
                 double *T, uint8_t *G,
                 int64_t *order, int64_t *n_order, uint8_t *tape)
{
    return march_run(nx, ny, nz, h3, speed, speed_const, width, T, G, order,
                     n_order, tape, 1);
}

int oracle_march_ho(int64_t nx, int64_t ny, int64_t nz, const double h3[3],
                    const double *speed, double speed_const, double width,
                    double *T, uint8_t *G,
                    int64_t *order, int64_t *n_order, int accuracy)
{
    if (accuracy != 1 && accuracy != 2)
        return -1;
    return march_run(nx, ny, nz, h3, speed, speed_const, width, T, G, order,
                     n_order, NULL, accuracy);
}

/* ------------------------------------------------------------------------ */
/* Fast sweeping with the textbook sorted Godunov update                      */
/* ------------------------------------------------------------------------ */

/* Unique t with sum_i max(t - a_i, 0)^2 / h_i^2 = s^2 for a1 <= a2 <= a3
 * (the values sorted with their cell sizes): take the first 1, 2 or 3 terms
 * while the root exceeds the next value.  With c_i = 1/h_i^2 the k-term
 * equation is (sum c) t^2 - 2 (sum c a) t + (sum c a^2) - s^2 = 0. */
static double godunov_sorted(const double a[3], const double hs[3], double s)
{
    double C = 0.0, B = 0.0, A2 = 0.0, t = OR_INF;
    for (int k = 0; k < 3; ++k) {
        if (a[k] == OR_INF || (k > 0 && t <= a[k]))
            break;
        double c = 1.0 / (hs[k] * hs[k]);
        C += c;
        B += c * a[k];
        A2 += c * a[k] * a[k];
        t = (B + sqrt(B * B - C * (A2 - s * s))) / C;
    }
    return t;
}

int oracle_fast_sweep(int64_t nx, int64_t ny, int64_t nz, const double h3[3],
                      const double *speed, double speed_const,
                      double *A, const uint8_t *fixed,
                      int64_t max_rounds, int64_t *rounds_out)
{
    grid_t g;
    if (grid_make(&g, nx, ny, nz) || !A || !fixed || !spacing_ok(h3))
        return -1;
    int64_t rounds = 0;
    for (; rounds < max_rounds;) {
        int changed = 0;
        for (int dirs = 0; dirs < 8; ++dirs) {
            int sx = (dirs & 1) ? -1 : 1, sy = (dirs & 2) ? -1 : 1,
                sz = (dirs & 4) ? -1 : 1;
            for (int64_t kk = 0; kk < nz; ++kk) {
                int64_t k = sz > 0 ? kk : nz - 1 - kk;
                for (int64_t jj = 0; jj < ny; ++jj) {
                    int64_t j = sy > 0 ? jj : ny - 1 - jj;
                    for (int64_t ii = 0; ii < nx; ++ii) {
                        int64_t i = sx > 0 ? ii : nx - 1 - ii;
                        int64_t p = (k * ny + j) * nx + i;
                        if (fixed[p])
                            continue;
                        double a[3], hs[3];
                        int64_t c[3] = {i, j, k};
                        for (int ax = 0; ax < 3; ++ax) {
                            double v = OR_INF;
                            int64_t qm = grid_nb(&g, p, c, ax, -1);
                            int64_t qp = grid_nb(&g, p, c, ax, +1);
                            if (qm >= 0 && A[qm] < v)
                                v = A[qm];
                            if (qp >= 0 && A[qp] < v)
                                v = A[qp];
                            a[ax] = v;
                            hs[ax] = h3[ax];
                        }
                        /* sort ascending, each cell size with its value */
                        for (int pass = 0; pass < 2; ++pass)
                            for (int q = 0; q < 2; ++q)
                                if (a[q] > a[q + 1]) {
                                    double t = a[q]; a[q] = a[q + 1]; a[q + 1] = t;
                                    t = hs[q]; hs[q] = hs[q + 1]; hs[q + 1] = t;
                                }
                        if (a[0] == OR_INF)
                            continue;
                        double F = speed_at(speed, speed_const, p);
                        double t = godunov_sorted(a, hs, 1.0 / F);
                        if (t < A[p]) {
                            A[p] = t;
                            changed = 1;
                        }
                    }
                }
            }
        }
        rounds += 1;
        if (!changed)
            break;
    }
    if (rounds_out)
        *rounds_out = rounds;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Linearisation about the final upwind sets (adjoint and tangent)            */
/* ------------------------------------------------------------------------ */

/* Upwind neighbours of p recorded in the tape: fills nbr[] (and their axes
 * in ax[]) and returns the count. */
static int tape_neighbours(const grid_t *g, int64_t p, uint8_t set,
                           int64_t nbr[3], int ax[3])
{
    int64_t c[3];
    grid_coord(g, p, c);
    int n = 0;
    for (int a = 0; a < 3; ++a) {
        int code = (set >> (2 * a)) & 3;
        if (code == 0)
            continue;
        int64_t q = grid_nb(g, p, c, a, code == 1 ? -1 : 1);
        if (q >= 0) {
            ax[n] = a;
            nbr[n++] = q;
        }
    }
    return n;
}

int oracle_adjoint(int64_t nx, int64_t ny, int64_t nz, const double h3[3],
                   const double *speed, double speed_const,
                   const double *T, const uint8_t *G, const uint8_t *tape,
                   const int64_t *order, int64_t n_order,
                   const double *dLdT, double *dLds, double *lambda)
{
    grid_t g;
    if (grid_make(&g, nx, ny, nz) || !T || !G || !tape || !order || !dLdT ||
        !dLds || !spacing_ok(h3))
        return -1;
    double *lam = lambda ? lambda
                         : (double *)malloc((size_t)g.n * sizeof(double));
    if (!lam)
        return -3;
    for (int64_t p = 0; p < g.n; ++p) {
        lam[p] = dLdT[p];
        dLds[p] = 0.0;
    }
    const double w[3] = {1.0 / (h3[0] * h3[0]), 1.0 / (h3[1] * h3[1]), 1.0 / (h3[2] * h3[2])};
    for (int64_t k = n_order - 1; k >= 0; --k) {
        int64_t p = order[k];
        if (G[p] == ORC_KNOWN_FIX)
            continue;
        int64_t nbr[3];
        int ax[3];
        int nn = tape_neighbours(&g, p, tape[p], nbr, ax);
        if (nn == 0)
            continue;
        double Tp = fabs(T[p]);
        double D = 0.0;
        for (int q = 0; q < nn; ++q)
            D += (Tp - fabs(T[nbr[q]])) * w[ax[q]];
        double sp = 1.0 / speed_at(speed, speed_const, p);
        dLds[p] = lam[p] * sp / D;
        for (int q = 0; q < nn; ++q)
            lam[nbr[q]] += lam[p] * (Tp - fabs(T[nbr[q]])) * w[ax[q]] / D;
    }
    if (!lambda)
        free(lam);
    return 0;
}

int oracle_tangent(int64_t nx, int64_t ny, int64_t nz, const double h3[3],
                   const double *speed, double speed_const,
                   const double *T, const uint8_t *G, const uint8_t *tape,
                   const int64_t *order, int64_t n_order,
                   const double *v, double *dT)
{
    grid_t g;
    if (grid_make(&g, nx, ny, nz) || !T || !G || !tape || !order || !v ||
        !dT || !spacing_ok(h3))
        return -1;
    for (int64_t p = 0; p < g.n; ++p)
        dT[p] = 0.0;
    const double w[3] = {1.0 / (h3[0] * h3[0]), 1.0 / (h3[1] * h3[1]), 1.0 / (h3[2] * h3[2])};
    for (int64_t k = 0; k < n_order; ++k) {
        int64_t p = order[k];
        if (G[p] == ORC_KNOWN_FIX)
            continue;
        int64_t nbr[3];
        int ax[3];
        int nn = tape_neighbours(&g, p, tape[p], nbr, ax);
        if (nn == 0)
            continue;
        double Tp = fabs(T[p]);
        double D = 0.0, acc = 0.0;
        for (int q = 0; q < nn; ++q) {
            double c = (Tp - fabs(T[nbr[q]])) * w[ax[q]];
            D += c;
            acc += c * dT[nbr[q]];
        }
        double sp = 1.0 / speed_at(speed, speed_const, p);
        dT[p] = (sp * v[p] + acc) / D;
    }
    return 0;
}
