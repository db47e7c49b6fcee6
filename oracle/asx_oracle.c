/*
 * asx_oracle.c -- plain FP64 CPU oracle of the explicit finite-volume step of the
 * porosity-extended Saint-Venant model on a regular hexagonal raster
 * (arxiv 2406.14933, "ASTERIX").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct statement of
 * what the GPU path computes.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark may load it.  It shares no code, header, table or
 * helper with the CUDA library; neither includes the other.
 *
 * What it follows (paper section / equation label):
 *   - model and forces:       Sec. 2.1, Eqs. swe_vegm_rm.02, eq_gforce, eq_tsa_darcy,
 *                             eq_tpa, eq_tau, eq_K_h_theta
 *   - cells and interfaces:   Sec. 2.2 (a)-(c), Eqs. fvm_2D_eq.06 (upwind mass),
 *                             fvm_2D_eq.05 (pressure-term mass), fvm_2D_eq.04
 *                             (interface velocity)
 *   - discrete operators:     Eq. fvm_2D_eq_frac.01 (J, S, L)
 *   - full discrete scheme:   Eq. fvm_2D_eq_frac.07, split as in Appendix A,
 *                             Eqs. fvm_2D_eq_frac.05-1/-2 (transport) and
 *                             fvm_2D_eq_frac.06-1/-2 (rain, then implicit friction)
 *   - time-step restriction:  Appendix A, Eqs. fvm_2D_eq_frac.12 and .13
 *   - implicit friction:      Appendix A, Eq. miu-formula
 *   - artificial viscosity:   Appendix A, Eqs. eq_artif_visc, eq_visc1 (optional)
 *   - linear soil resistance: Sec. 4 (Thacker's problem), Eq. eq_soil_friction_thacker
 *                             (optional, tau = 0 by default)
 *   - rain:                   Appendix C (piecewise-linear hyetograph)
 *   - boundary types:         Sec. 3 "Data In" (free discharge default, wall, given
 *                             mass flux) and Sec. 4, Eq. numerics-bc (Dirichlet)
 *
 * Readings of points the paper leaves open (each is listed in the design notes):
 *   - raster: pointy-top hexagons in rows along x, every row `cols` cells long, odd
 *     rows shifted east by half a centre spacing; "radius" l = edge length =
 *     circumradius, so sigma = (3 sqrt3 / 2) l^2, centre spacing sqrt3 l, and the
 *     normal of the edge shared with a neighbour is the unit vector towards it.
 *   - prognostic mass m = theta*h; the rain source M is the rain rate r(t) itself
 *     (independent of theta), evaluated at t^{n+1} as printed.
 *   - phi_min = sigma / (6 l): the perimeter of a cell counts all six sides.
 *   - wall edge: mirror ghost, so v_n = 0 and w_j = w_i; the edge adds nothing.
 *     free-discharge edge: ghost copy of the inner cell, outflow only:
 *     F = l m_i max(v_i.n, 0), momentum flux F v_i, no pressure term.
 *   - dry cell: m == 0 exactly; if the friction denominator is 0, v = 0.
 *   - m < 0 after the update (only possible through rounding or CFL > 1) is set
 *     to 0 and the water so created is booked in the ledger as "clamped".
 *   - boundary edge side: a neighbour row outside [0,rows) puts the edge on the
 *     S or N side; otherwise a column outside [0,cols) puts it on W or E.  A side may
 *     restrict free discharge to an interval of positions (an outlet); the rest of
 *     that side is a wall.
 *   - dt_n = min(dt_max, CFL phi / c_max^n) (dt_max if c_max = 0), cut so that a
 *     step never passes t_end or the next hydrograph sample time.
 *
 * Everything is double precision, one cell at a time, each operator summed over the
 * neighbours of the cell exactly as written.  Built plainly the file is single-threaded;
 * built with OpenMP (-fopenmp) the rows of a step are shared among threads.  A cell's
 * update reads only the state at t^n and writes only its own outputs, and the step's
 * outflow and clamp sums are formed after the cell loop, cell by cell in row-major
 * order as the single-threaded loop adds them, so both builds give the same bits.
 */
#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_W 0
#define ORC_E 1
#define ORC_S 2
#define ORC_N 3
#define ORC_WALL 0
#define ORC_FREE 1
#define ORC_FLUX 2          /* given mass flux (Sec. 3, boundary conditions) */
#define ORC_DIRICHLET 3     /* given depth and velocity (Sec. 4, Eq. numerics-bc) */

typedef struct {
    int rows, cols;
    double l;               /* edge length ("radius") [m] */
    int bc[4];              /* boundary type per side W, E, S, N */
    int free_begin[4];      /* free discharge applies for positions in [begin, end) along */
    int free_end[4];        /* the side (column for S/N, row for W/E); begin == end: all */
    double g;               /* gravity [m/s^2] */
    double cfl;             /* Courant number in (0, 1] */
    double dt_max;          /* maximum time step [s] */
    const double *z;        /* bed elevation per cell [m] */
    const double *theta;    /* porosity per cell, (0, 1] */
    const double *alpha_s;  /* soil friction coefficient per cell [-] */
    const double *alpha_p;  /* plant drag coefficient per cell [1/m] */
    int n_rain;             /* hyetograph points (0 = no rain) */
    const double *rain_t;   /* [s], increasing */
    const double *rain_r;   /* [m/s] */
    int viscosity;          /* 1 = add the artificial viscosity flux */
    double tau;             /* linear soil resistance -tau h v [1/s] of Thacker's problem
                               (Sec. 4, Eq. eq_soil_friction_thacker); 0 = none */
    double h_dry;           /* depth [m] below which a cell's velocity is set to zero after
                               the friction step; 0 = none (dry means m = 0 exactly) */
    double bc_q[4];         /* ORC_FLUX: inflow per unit length of the side [m^2/s] */
    double bc_h[4];         /* ORC_DIRICHLET: ghost depth [m] */
    double bc_u[4];         /* ORC_DIRICHLET: ghost speed along the inward normal [m/s] */
} orc_problem;

typedef struct {
    double rain_in;   /* sum over steps of sigma * dt * r(t^{n+1}) over all cells [m^3] */
    double outflow;   /* volume that left through free-discharge edges [m^3] */
    double clamped;   /* volume created by setting negative masses to zero [m^3] */
    long long steps;
} orc_ledger;

/* ---------------- geometry of the hexagonal raster (Sec. 2.2 (a)) ---------------- */

/* Directions 0..5 point E, NE, NW, W, SW, SE; the unit normal of direction d is
 * (cos 60d deg, sin 60d deg). */
static void orc_normal(int d, double *n1, double *n2)
{
    const double s = sqrt(3.0) / 2.0;
    static const double c1[6] = {1.0, 0.5, -0.5, -1.0, -0.5, 0.5};
    static const int sg[6] = {0, 1, 1, 0, -1, -1};
    *n1 = c1[d];
    *n2 = sg[d] * s;
}

/* Neighbour of cell (r, c) in direction d.  Returns 1 and the neighbour's index if
 * it lies in the raster; otherwise 0 and the boundary side of the shared edge. */
int orc_neighbour(int rows, int cols, int r, int c, int d, int *j, int *side)
{
    int odd = r & 1, rr = r, cc = c;
    switch (d) {
    case 0: cc = c + 1; break;
    case 3: cc = c - 1; break;
    case 1: rr = r + 1; cc = odd ? c + 1 : c; break;
    case 2: rr = r + 1; cc = odd ? c : c - 1; break;
    case 4: rr = r - 1; cc = odd ? c : c - 1; break;
    case 5: rr = r - 1; cc = odd ? c + 1 : c; break;
    }
    if (rr < 0) { *side = ORC_S; return 0; }
    if (rr >= rows) { *side = ORC_N; return 0; }
    if (cc < 0) { *side = ORC_W; return 0; }
    if (cc >= cols) { *side = ORC_E; return 0; }
    *j = rr * cols + cc;
    return 1;
}

/* Boundary type of the edge of cell (r, c) on `side`: the side's type inside its interval
 * [free_begin, free_end) of positions (all of it when begin == end), a wall outside. */
static int orc_bc_at(const orc_problem *p, int side, int r, int c)
{
    int pos = (side == ORC_S || side == ORC_N) ? c : r;
    if (p->free_begin[side] == p->free_end[side]) return p->bc[side];
    return (pos >= p->free_begin[side] && pos < p->free_end[side]) ? p->bc[side] : ORC_WALL;
}

double orc_sigma(double l) { return 1.5 * sqrt(3.0) * l * l; }

/* phi = sigma_i / sum_j l_(i,j) with all six sides of the cell (Eq. fvm_2D_eq_frac.13). */
double orc_phi(double l) { return orc_sigma(l) / (6.0 * l); }

/* Threads the cell loops use: sets the count when n > 0, returns the count in force
 * (always 1 in the single-threaded build). */
int orc_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* ---------------- forcing ---------------- */

/* Piecewise-linear hyetograph r(t), zero outside [t_0, t_last] (Appendix C gives the
 * triangular case; the table form also carries constant and multi-peak storms). */
double orc_rain_rate(const orc_problem *p, double t)
{
    int k;
    if (p->n_rain <= 0) return 0.0;
    if (t < p->rain_t[0] || t > p->rain_t[p->n_rain - 1]) return 0.0;
    if (p->n_rain == 1) return p->rain_r[0];
    for (k = 0; k + 1 < p->n_rain; k++) {
        double t0 = p->rain_t[k], t1 = p->rain_t[k + 1];
        if (t <= t1) {
            if (t1 == t0) return p->rain_r[k + 1];
            return p->rain_r[k] + (p->rain_r[k + 1] - p->rain_r[k]) * (t - t0) / (t1 - t0);
        }
    }
    return p->rain_r[p->n_rain - 1];
}

/* Resistance coefficient K(h, theta) = alpha_p h (1 - theta) + theta alpha_s
 * (Eqs. eq_tau, eq_K_h_theta with the Darcy-Weisbach soil term eq_tsa_darcy). */
static double orc_K(const orc_problem *p, int i, double h)
{
    return p->alpha_p[i] * h * (1.0 - p->theta[i]) + p->theta[i] * p->alpha_s[i];
}

/* Closed-form solution of  alpha v + beta |v| v = gamma  (Appendix A, Eq. miu-formula):
 * v = mu gamma with mu = 2 / (alpha + sqrt(alpha^2 + 4 beta |gamma|)); v = 0 when the
 * denominator vanishes (dry cell without friction). */
void orc_friction(double alpha, double beta, double g1, double g2, double *v1, double *v2)
{
    /* |gamma| without underflow of the squares, and v = 2 gamma / den rather than
     * (2 / den) gamma, so that films of subnormal depth give finite velocities */
    double ng = hypot(g1, g2);
    double den = alpha + sqrt(alpha * alpha + 4.0 * beta * ng);
    if (den > 0.0) {
        *v1 = 2.0 * g1 / den;
        *v2 = 2.0 * g2 / den;
    } else {
        *v1 = 0.0;
        *v2 = 0.0;
    }
}

/* ---------------- time step (Appendix A, Eqs. fvm_2D_eq_frac.12-13) ---------------- */

/* c_max = max_i |v_i| + sqrt(g h_i), h_i = m_i / theta_i. */
double orc_cmax(const orc_problem *p, const double *m, const double *v1, const double *v2)
{
    int n = p->rows * p->cols, i;
    double cmax = 0.0;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) reduction(max : cmax)
#endif
    for (i = 0; i < n; i++) {
        double h = m[i] / p->theta[i];
        double c = sqrt(v1[i] * v1[i] + v2[i] * v2[i]) + sqrt(p->g * h);
        if (c > cmax) cmax = c;
    }
    return cmax;
}

/* tau_n = CFL phi_min / c_max; dt_max when the raster is at rest. */
double orc_cfl_dt(const orc_problem *p, const double *m, const double *v1, const double *v2)
{
    double cmax = orc_cmax(p, m, v1, v2);
    double dt = p->dt_max;
    if (cmax > 0.0) {
        double tau = p->cfl * orc_phi(p->l) / cmax;
        if (tau < dt) dt = tau;
    }
    return dt;
}

/* ---------------- one time step ---------------- */

/* Advance (m, v1, v2) at t^n by dt to t_next = t^{n+1}.  Outputs may not alias inputs.
 * Returns 0, or -1 on a non-finite result (or when the step's scratch cannot be
 * allocated). */
static int orc_step_ws(const orc_problem *p, const double *m, const double *v1, const double *v2,
                       double dt, double t_next, double *m_out, double *v1_out, double *v2_out,
                       orc_ledger *led, double *cell_out, double *cell_clamp);

int orc_step(const orc_problem *p, const double *m, const double *v1, const double *v2,
             double dt, double t_next,
             double *m_out, double *v1_out, double *v2_out, orc_ledger *led)
{
    const size_t n = (size_t)p->rows * (size_t)p->cols;
    double *cell_out = (double *)malloc(sizeof(double) * n);
    double *cell_clamp = (double *)malloc(sizeof(double) * n);
    int rc = -1;
    if (cell_out && cell_clamp)
        rc = orc_step_ws(p, m, v1, v2, dt, t_next, m_out, v1_out, v2_out, led, cell_out, cell_clamp);
    free(cell_out);
    free(cell_clamp);
    return rc;
}

/* orc_step with caller-provided scratch for the per-cell outflow rates and clamped
 * volumes (n doubles each). */
static int orc_step_ws(const orc_problem *p, const double *m, const double *v1, const double *v2,
                       double dt, double t_next, double *m_out, double *v1_out, double *v2_out,
                       orc_ledger *led, double *cell_out, double *cell_clamp)
{
    const int rows = p->rows, cols = p->cols, n = rows * cols;
    const double l = p->l, g = p->g;
    const double sigma = orc_sigma(l);
    const double rain = orc_rain_rate(p, t_next);   /* M_i(t^{n+1}) = r(t^{n+1}) */
    double out_rate_total = 0.0, clamp_total = 0.0;
    /* per-cell outflow rate and clamped volume (cell_out, cell_clamp), summed after the
     * cell loop */
    int r, i, bad = 0;

#ifdef _OPENMP
#pragma omp parallel for schedule(static) reduction(| : bad)
#endif
    for (r = 0; r < rows; r++) {
        int c, d;
        for (c = 0; c < cols; c++) {
            const int i = r * cols + c;
            const double hi = m[i] / p->theta[i];
            const double ci = sqrt(v1[i] * v1[i] + v2[i] * v2[i]) + sqrt(g * hi);
            double L = 0.0, J1 = 0.0, J2 = 0.0, S1 = 0.0, S2 = 0.0;
            double out_rate = 0.0;

            for (d = 0; d < 6; d++) {
                double n1, n2;
                int j, side;
                orc_normal(d, &n1, &n2);
                if (orc_neighbour(rows, cols, r, c, d, &j, &side)) {
                    const double hj = m[j] / p->theta[j];
                    /* Eq. fvm_2D_eq.04: interface velocity and its normal component */
                    const double vb1 = (v1[i] + v1[j]) / 2.0;
                    const double vb2 = (v2[i] + v2[j]) / 2.0;
                    const double vn = vb1 * n1 + vb2 * n2;
                    /* Eq. eq_gforce: w = g (z + h); w_j - w_i */
                    const double dw = g * ((p->z[j] - p->z[i]) + (hj - hi));
                    /* Eq. fvm_2D_eq.06: upwind theta*h (irrelevant when v_n = 0) */
                    double thh = 0.0, hat;
                    if (vn > 0.0) thh = m[i];
                    else if (vn < 0.0) thh = m[j];
                    /* Eq. fvm_2D_eq.05: theta*h used by the pressure term */
                    if (vn != 0.0) hat = thh;
                    else hat = (dw < 0.0) ? m[i] : m[j];   /* w_i > w_j -> i, else j */
                    /* Eq. fvm_2D_eq_frac.01 */
                    L -= l * thh * vn;
                    J1 -= l * thh * vb1 * vn;
                    J2 -= l * thh * vb2 * vn;
                    S1 -= 0.5 * l * dw * hat * n1;
                    S2 -= 0.5 * l * dw * hat * n2;
                    if (p->viscosity) {
                        /* Eqs. eq_artif_visc, eq_visc1: l c_(i,j) mu_(i,j) (v_j - v_i),
                         * harmonic mean mu with 0/0 taken as 0 */
                        const double cj = sqrt(v1[j] * v1[j] + v2[j] * v2[j]) + sqrt(g * hj);
                        const double cij = ci > cj ? ci : cj;
                        const double den = m[i] + m[j];
                        const double mu = den > 0.0 ? 2.0 * m[i] * m[j] / den : 0.0;
                        J1 += l * cij * mu * (v1[j] - v1[i]);
                        J2 += l * cij * mu * (v2[j] - v2[i]);
                    }
                } else {
                    const int bt = orc_bc_at(p, side, r, c);
                    /* outward unit normal of the side */
                    const double ns1 = side == ORC_W ? -1.0 : side == ORC_E ? 1.0 : 0.0;
                    const double ns2 = side == ORC_S ? -1.0 : side == ORC_N ? 1.0 : 0.0;
                    if (bt == ORC_FREE) {
                        /* free discharge: ghost = copy of cell i, outflow only */
                        const double vn = v1[i] * n1 + v2[i] * n2;
                        if (vn > 0.0) {
                            L -= l * m[i] * vn;
                            J1 -= l * m[i] * v1[i] * vn;
                            J2 -= l * m[i] * v2[i] * vn;
                            out_rate += l * m[i] * vn;
                        }
                    } else if (bt == ORC_FLUX && p->bc_q[side] > 0.0) {
                        /* given mass flux q along the inward side normal: the edge admits
                         * l q (n_side . n); the water enters with speed q / h, h the
                         * cell's depth but at least the critical depth (q^2 / g)^(1/3);
                         * the ghost's surface is the cell's, so no pressure term */
                        const double q = p->bc_q[side];
                        const double qin = l * q * (ns1 * n1 + ns2 * n2);
                        const double hc = cbrt(q * q / g);
                        const double uin = q / (hi > hc ? hi : hc);
                        L += qin;
                        J1 += qin * uin * (-ns1);
                        J2 += qin * uin * (-ns2);
                        out_rate -= qin;
                    } else if (bt == ORC_DIRICHLET) {
                        /* given depth and velocity: a ghost cell on cell i's bed and
                         * porosity with h = h_b and v = -u_b n_side, through the same
                         * edge formulas as an interior neighbour (no viscosity) */
                        const double hg = p->bc_h[side], mg = p->theta[i] * hg;
                        const double vg1 = -p->bc_u[side] * ns1, vg2 = -p->bc_u[side] * ns2;
                        const double vb1 = (v1[i] + vg1) / 2.0;
                        const double vb2 = (v2[i] + vg2) / 2.0;
                        const double vn = vb1 * n1 + vb2 * n2;
                        const double dw = g * (hg - hi);
                        double thh = 0.0, hat;
                        if (vn > 0.0) thh = m[i];
                        else if (vn < 0.0) thh = mg;
                        if (vn != 0.0) hat = thh;
                        else hat = (dw < 0.0) ? m[i] : mg;
                        L -= l * thh * vn;
                        J1 -= l * thh * vb1 * vn;
                        J2 -= l * thh * vb2 * vn;
                        S1 -= 0.5 * l * dw * hat * n1;
                        S2 -= 0.5 * l * dw * hat * n2;
                        out_rate += l * thh * vn;
                    }
                    /* wall: mirror ghost, v_n = 0 and w_j = w_i, nothing to add */
                }
            }

            {
                /* Eq. fvm_2D_eq_frac.05-1: transport of theta*h */
                const double m_star = m[i] + dt / sigma * L;
                /* Eq. fvm_2D_eq_frac.06-1: rain at t^{n+1} (explicit, M does not depend on h) */
                double m_new = m_star + dt * rain;
                /* Eq. fvm_2D_eq_frac.05-2: transport of theta*h*v plus the surface-gradient force */
                const double g1 = m[i] * v1[i] + dt / sigma * (J1 + S1);
                const double g2 = m[i] * v2[i] + dt / sigma * (J2 + S2);
                double h_new, beta;
                cell_clamp[i] = 0.0;
                if (m_new < 0.0) {
                    cell_clamp[i] = -m_new * sigma;
                    m_new = 0.0;
                }
                /* Eq. fvm_2D_eq_frac.06-2 via Eq. miu-formula; a linear resistance
                 * -tau h v, taken implicitly like the rest, adds dt tau h^{n+1} to alpha:
                 * (theta h + dt tau h) v + beta |v| v = gamma */
                h_new = m_new / p->theta[i];
                beta = dt * orc_K(p, i, h_new);
                m_out[i] = m_new;
                orc_friction(m_new + dt * p->tau * h_new, beta, g1, g2, &v1_out[i], &v2_out[i]);
                if (h_new < p->h_dry) {
                    v1_out[i] = 0.0;
                    v2_out[i] = 0.0;
                }
                if (!isfinite(m_new) || !isfinite(v1_out[i]) || !isfinite(v2_out[i])) bad = 1;
            }
            cell_out[i] = out_rate;
        }
    }
    /* the step's sums, in row-major order (adding a cell's 0 leaves a sum unchanged) */
    for (i = 0; i < n; i++) {
        out_rate_total += cell_out[i];
        clamp_total += cell_clamp[i];
    }
    if (led) {
        led->rain_in += sigma * dt * rain * (double)n;
        led->outflow += dt * out_rate_total;
        led->clamped += clamp_total;
        led->steps += 1;
    }
    return bad ? -1 : 0;
}

/* Water volume sum_i sigma theta_i h_i. */
double orc_storage(const orc_problem *p, const double *m)
{
    int n = p->rows * p->cols, i;
    double s = 0.0;
    for (i = 0; i < n; i++) s += m[i];
    return s * orc_sigma(p->l);
}

/* ---------------- time loop ---------------- */

/* Run from *t to t_end (or max_steps), updating m, v1, v2 and *t in place.
 * If t_replay is given, step k ends at t_replay[k] instead of the CFL choice.
 * If sample_dt > 0, every step is cut at the sample times k*sample_dt and the
 * cumulative outflow at each sample time is written to samples[] (cap entries).
 * Returns the number of steps taken, or -1 on a non-finite state. */
long long orc_run(const orc_problem *p, double *m, double *v1, double *v2, double *t,
                  double t_end, long long max_steps, const double *t_replay, long long n_replay,
                  double sample_dt, double *samples, int cap, int *n_samples, orc_ledger *led)
{
    const int n = p->rows * p->cols;
    /* one workspace: the other state buffers and the step's per-cell scratch; the
     * state moves between the caller's arrays and these by swapping pointers */
    double *ws = (double *)malloc(sizeof(double) * (size_t)n * 5);
    double *cm = m, *ca = v1, *cb = v2;
    double *m2, *a2, *b2;
    long long k = 0;
    int ns = n_samples ? *n_samples : 0;
    int rc = 0;
    if (!ws) return -1;
    m2 = ws;
    a2 = ws + (size_t)n;
    b2 = ws + 2 * (size_t)n;

    while (*t < t_end && k < max_steps) {
        double t_next, dt;
        double next_sample = 0.0;
        if (sample_dt > 0.0) next_sample = (double)(ns + 1) * sample_dt;
        if (t_replay) {
            if (k >= n_replay) break;
            t_next = t_replay[k];
            dt = t_next - *t;
        } else {
            double t_stop = t_end;
            dt = orc_cfl_dt(p, cm, ca, cb);
            if (sample_dt > 0.0 && next_sample < t_stop) t_stop = next_sample;
            if (*t + dt >= t_stop) {
                dt = t_stop - *t;
                t_next = t_stop;
            } else {
                t_next = *t + dt;
            }
        }
        rc = orc_step_ws(p, cm, ca, cb, dt, t_next, m2, a2, b2, led, ws + 3 * (size_t)n, ws + 4 * (size_t)n);
        {
            double *x;
            x = cm; cm = m2; m2 = x;
            x = ca; ca = a2; a2 = x;
            x = cb; cb = b2; b2 = x;
        }
        *t = t_next;
        k++;
        if (sample_dt > 0.0 && t_next == next_sample) {
            if (samples && ns < cap) samples[ns] = led ? led->outflow : 0.0;
            ns++;
        }
        if (rc) break;
    }
    if (n_samples) *n_samples = ns;
    if (cm != m) {   /* the state ended in the workspace: copy it to the caller's arrays */
        memcpy(m, cm, sizeof(double) * (size_t)n);
        memcpy(v1, ca, sizeof(double) * (size_t)n);
        memcpy(v2, cb, sizeof(double) * (size_t)n);
    }
    free(ws);
    return rc ? -1 : k;
}
