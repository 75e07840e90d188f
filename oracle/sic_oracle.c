/*
 * sic_oracle.c -- plain FP64 CPU oracle of the simplex-in-cell (SIC) step for
 * the 1D periodic Vlasov-Poisson system (Kates-Harbeck, Totorica, Zrake & Abel,
 * arXiv:1506.07207).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link or call this
 * file: only the tests, the package's smoke check and the benchmark's CPU
 * baseline leg use it.  It shares no code, header, table or helper with the
 * CUDA path.  It is deliberately slow and literal: every function is one of the
 * paper's definitions written out as plain loops in double precision, with no
 * blocking, fusion, fixed point or reordering.
 *
 * Conventions (the paper leaves these open; the readings used are):
 *   - Units: C = 1 in the Poisson equation of Sec. 2.1, so with E = -dPhi/dx
 *     the field obeys dE/dx = rho and a tracer accelerates by qm * E
 *     (qm = charge-to-mass factor, +1 in the paper's sign convention).
 *   - rho = n - mean(n): the neutralising background is the computed mean
 *     density (Sec. 2.1, "mean density is set to zero").
 *   - Mesh: cell j covers [j dx, (j+1) dx), left-closed; rho is a cell
 *     average (Eq. rho_sum with V~ = dx); E lives on the nodes x_j = j dx and
 *     is the exact integral of rho from node to node, shifted to zero mean
 *     (periodic potential).
 *   - Segment charge q_s = (w_i + w_{i+1}) / 2 (Sec. 2.5 uses the mean of the
 *     two tracer charges; for equal tracer weights it is the tracer weight).
 *   - A segment of zero length puts its whole charge in the cell holding its
 *     point (the footnote of Sec. 2.3 only asks that charge be kept).
 *   - Closed sheets close with the segment (x_N, x_1 + winding * L): the
 *     periodic identification x_{N+1} = x_1 of Sec. 2.3 taken on the unwrapped
 *     line.
 *   - Time integration (not stated in the paper): leapfrog kick-drift,
 *     v^{n+1/2} = v^{n-1/2} + dt qm E^n(x^n), x^{n+1} = x^n + dt v^{n+1/2}.
 *   - Gather: linear weighting between the two nodes around a tracer
 *     (Sec. 2.3, end: forces gathered "using linear weighting").
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Periodic reduction of an (unbounded) cell number into [0, nx). */
static int wrap_cell(long m, int nx)
{
    long r = m % (long)nx;
    if (r < 0)
        r += nx;
    return (int)r;
}

/*
 * Charge of one box-function particle spread over the cells it overlaps.
 *
 * Sec. 2.3: the particle between tracers at xa and xb is the box function
 * b(x) = 1/|xa - xb| on (min, max); Eq. overlap gives its overlap with cell j
 * as the integral of b over the cell, and Eq. rho_sum weights that overlap by
 * the particle's charge q.  With periodic boundaries every image of a cell
 * counts, so the loop runs over the unwrapped cells m touched by [a, b] and
 * folds m into [0, nx).  The clip is taken in physical units; cells one past
 * each end are visited too so that rounding of a/dx or b/dx cannot lose a cell
 * (their clipped length is then <= 0 and they are skipped).
 */
static void deposit_segment(double xa, double xb, double q, int nx, double dx,
                            double *charge)
{
    double a = xa < xb ? xa : xb;
    double b = xa < xb ? xb : xa;
    long ma = (long)floor(a / dx);
    long mb = (long)floor(b / dx);
    if (b == a) {
        charge[wrap_cell(ma, nx)] += q;
        return;
    }
    double len = b - a;
    for (long m = ma - 1; m <= mb + 1; ++m) {
        double lo = a > m * dx ? a : m * dx;
        double hi = b < (m + 1) * dx ? b : (m + 1) * dx;
        if (hi > lo)
            charge[wrap_cell(m, nx)] += q * (hi - lo) / len;
    }
}

/*
 * Total charge per cell of all sheets (Eq. rho_sum times the cell volume).
 *
 * A sheet is an ordered run of tracers (Sec. 2.2, "Implications of the Sheet
 * Topology"); every adjacent pair is a particle (Sec. 2.3).  counts[s] tracers
 * of sheet s follow each other in x[] and w[].  closed[s] != 0 adds the
 * closing particle (last, first + winding[s] * L).
 * Returns 0, or -1 for a sheet with fewer than two tracers.
 */
int orc_deposit(int nx, double L, int n_sheets, const int32_t *counts,
                const uint8_t *closed, const int32_t *winding,
                const double *x, const double *w, double *charge)
{
    double dx = L / nx;
    memset(charge, 0, sizeof(double) * (size_t)nx);
    long base = 0;
    for (int s = 0; s < n_sheets; ++s) {
        long n = counts[s];
        if (n < 2)
            return -1;
        for (long i = 0; i + 1 < n; ++i) {
            double q = 0.5 * (w[base + i] + w[base + i + 1]);
            deposit_segment(x[base + i], x[base + i + 1], q, nx, dx, charge);
        }
        if (closed[s]) {
            double q = 0.5 * (w[base + n - 1] + w[base]);
            double xb = x[base] + (double)winding[s] * L;
            deposit_segment(x[base + n - 1], xb, q, nx, dx, charge);
        }
        base += n;
    }
    return 0;
}

/*
 * The same deposit with the particles' charges given directly: qseg[i] is the
 * charge of the particle that starts at tracer i (for the last tracer of a
 * closed sheet, the closing particle; ignored for the last tracer of an open
 * sheet).  Refinement (Sec. 2.6) splits particles and halves their charges,
 * which tracer weights cannot express, so a refined sheet carries its charge
 * on the particles, as Sec. 2.3 defines it.
 */
int orc_deposit_seg(int nx, double L, int n_sheets, const int32_t *counts,
                    const uint8_t *closed, const int32_t *winding,
                    const double *x, const double *qseg, double *charge)
{
    double dx = L / nx;
    memset(charge, 0, sizeof(double) * (size_t)nx);
    long base = 0;
    for (int s = 0; s < n_sheets; ++s) {
        long n = counts[s];
        if (n < 2)
            return -1;
        for (long i = 0; i + 1 < n; ++i)
            deposit_segment(x[base + i], x[base + i + 1], qseg[base + i], nx, dx, charge);
        if (closed[s])
            deposit_segment(x[base + n - 1], x[base] + (double)winding[s] * L, qseg[base + n - 1], nx, dx,
                            charge);
        base += n;
    }
    return 0;
}

/*
 * Piecewise-linear particles (Sec. 2.5, Eq. piecewise_linear with the
 * gradient of Eq. gradient_rho_estimate).
 *
 * Particle s between tracers x_i and x_{i+1} keeps its charge q_s and its
 * zeroth-order density rho0_s = q_s / |x_{i+1} - x_i|, centred on its centroid
 * c_s = (x_i + x_{i+1}) / 2; on its extent the density is
 *     rho0_s + (x - c_s) g_s,
 * with g_s the central difference over the two particles next to it along
 * the sheet:
 *     g_s = (rho0_{s+1} - rho0_{s-1}) / (c_{s+1} - c_{s-1}).
 * g_s is 0 (the particle stays a box) when a neighbour is missing (the two
 * ends of an open sheet), when any of the three particles has zero length,
 * or when the centroids are not in order along the sheet, i.e. neither
 * c_{s-1} < c_s < c_{s+1} nor the reverse (the corner of a fold, Sec. 2.5).
 * On a closed sheet the closing particle (x_{n-1}, x_0 + winding L) is the
 * neighbour of the first and the last ones; its centroid is shifted by one
 * winding when it is compared with theirs.  A particle at least one box
 * length long also stays a box: Sec. 3.2 notes that a run cannot go on
 * once a particle outgrows the box (it no longer describes the phase-space
 * sheet), and a linear profile about the centroid of such a particle would
 * overlap its own periodic image, so the uniform density of Sec. 2.3 is kept.
 *
 * The charge of the piece [lo, hi] of a particle inside a cell is the integral
 * of its density: rho0 (hi - lo) + g ((hi - c)^2 - (lo - c)^2) / 2, summed over
 * the periodic images like deposit_segment.  Over the whole particle the
 * linear term integrates to zero, so every particle still carries exactly q.
 */
static void deposit_linear_segment(double xa, double xb, double q, double g,
                                   int nx, double dx, double *charge)
{
    double a = xa < xb ? xa : xb;
    double b = xa < xb ? xb : xa;
    long ma = (long)floor(a / dx);
    long mb = (long)floor(b / dx);
    if (b == a) {
        charge[wrap_cell(ma, nx)] += q;
        return;
    }
    double rho0 = q / (b - a);
    double c = 0.5 * (a + b);
    for (long m = ma - 1; m <= mb + 1; ++m) {
        double lo = a > m * dx ? a : m * dx;
        double hi = b < (m + 1) * dx ? b : (m + 1) * dx;
        if (hi > lo)
            charge[wrap_cell(m, nx)] +=
                rho0 * (hi - lo) + g * ((hi - c) * (hi - c) - (lo - c) * (lo - c)) / 2.0;
    }
}

/* w (tracer weights) or qseg (per-particle charges, as for orc_deposit_seg):
 * exactly one of them is given. */
static int deposit_linear_sheets(int nx, double L, int n_sheets, const int32_t *counts,
                                 const uint8_t *closed, const int32_t *winding,
                                 const double *x, const double *w, const double *qseg,
                                 double *charge)
{
    double dx = L / nx;
    memset(charge, 0, sizeof(double) * (size_t)nx);
    long base = 0;
    for (int s = 0; s < n_sheets; ++s) {
        long n = counts[s];
        if (n < 2)
            return -1;
        /* the sheet's particles: endpoints, charge, density, centroid */
        long np = closed[s] ? n : n - 1;
        double *xa = (double *)malloc(sizeof(double) * (size_t)np);
        double *xb = (double *)malloc(sizeof(double) * (size_t)np);
        double *q = (double *)malloc(sizeof(double) * (size_t)np);
        double *rho0 = (double *)malloc(sizeof(double) * (size_t)np);
        double *c = (double *)malloc(sizeof(double) * (size_t)np);
        double shift = (double)winding[s] * L;
        for (long k = 0; k < np; ++k) {
            long i = k, j = k + 1;
            xa[k] = x[base + i];
            if (j < n) {
                xb[k] = x[base + j];
                q[k] = qseg ? qseg[base + i] : 0.5 * (w[base + i] + w[base + j]);
            } else {
                xb[k] = x[base] + shift;
                q[k] = qseg ? qseg[base + i] : 0.5 * (w[base + i] + w[base]);
            }
            double len = fabs(xb[k] - xa[k]);
            rho0[k] = len > 0.0 ? q[k] / len : 0.0;
            c[k] = 0.5 * (xa[k] + xb[k]);
        }
        for (long k = 0; k < np; ++k) {
            double g = 0.0;
            int has_prev = closed[s] || k > 0;
            int has_next = closed[s] || k + 1 < np;
            if (has_prev && has_next) {
                long kp = k > 0 ? k - 1 : np - 1;
                long kn = k + 1 < np ? k + 1 : 0;
                double cp = c[kp] - (k == 0 ? shift : 0.0);
                double cn = c[kn] + (k + 1 == np ? shift : 0.0);
                int lengths = xa[kp] != xb[kp] && xa[k] != xb[k] && xa[kn] != xb[kn];
                int ordered = (cp < c[k] && c[k] < cn) || (cp > c[k] && c[k] > cn);
                int shorter = fabs(xb[k] - xa[k]) < L;
                if (lengths && ordered && shorter)
                    g = (rho0[kn] - rho0[kp]) / (cn - cp);
            }
            deposit_linear_segment(xa[k], xb[k], q[k], g, nx, dx, charge);
        }
        free(xa);
        free(xb);
        free(q);
        free(rho0);
        free(c);
        base += n;
    }
    return 0;
}

/*
 * PIC deposits of the tracers themselves, for the comparison runs of Sec. 3
 * (Sec. 2.4 gives the weightings): every tracer is a point charge w_i.
 *   scheme 2, zero order (nearest grid point): the whole charge goes to the
 *     cell holding the tracer (the cell whose centre is nearest);
 *   scheme 3, first order (cloud in cell): the charge is shared between the
 *     two cells whose centres (j + 1/2) dx bracket the tracer, linearly in
 *     its distance to each centre.
 */
int orc_deposit_pic(int nx, double L, long n_tracers, const double *x,
                    const double *w, int scheme, double *charge)
{
    double dx = L / nx;
    memset(charge, 0, sizeof(double) * (size_t)nx);
    for (long i = 0; i < n_tracers; ++i) {
        if (scheme == 2) {
            charge[wrap_cell((long)floor(x[i] / dx), nx)] += w[i];
        } else {
            double p = x[i] / dx - 0.5;
            double m = floor(p);
            double f = p - m;
            charge[wrap_cell((long)m, nx)] += w[i] * (1.0 - f);
            charge[wrap_cell((long)m + 1, nx)] += w[i] * f;
        }
    }
    return 0;
}

int orc_deposit_linear(int nx, double L, int n_sheets, const int32_t *counts,
                       const uint8_t *closed, const int32_t *winding,
                       const double *x, const double *w, double *charge)
{
    return deposit_linear_sheets(nx, L, n_sheets, counts, closed, winding, x, w, NULL, charge);
}

/* Piecewise-linear particles with per-particle charges (refined sheets). */
int orc_deposit_linear_seg(int nx, double L, int n_sheets, const int32_t *counts,
                           const uint8_t *closed, const int32_t *winding,
                           const double *x, const double *qseg, double *charge)
{
    return deposit_linear_sheets(nx, L, n_sheets, counts, closed, winding, x, NULL, qseg, charge);
}

/* The deposit of the given kind: 0 box particles (Sec. 2.3), 1 piecewise
 * linear particles (Sec. 2.5), 2 and 3 PIC point charges (NGP, CIC). */
int orc_moments(int nx, double L, int n_sheets, const int32_t *counts,
                const uint8_t *closed, const int32_t *winding, const double *x,
                const double *v, const double *w, int weighting, double *n,
                double *j);
int orc_deposit_first(int nx, double L, int n_sheets, const int32_t *counts,
                      const uint8_t *closed, const int32_t *winding,
                      const double *x, const double *w, double *charge);

static int deposit_order(int order, int nx, double L, int n_sheets,
                         const int32_t *counts, const uint8_t *closed,
                         const int32_t *winding, const double *x,
                         const double *w, double *charge)
{
    if (order == 4)
        return orc_deposit_first(nx, L, n_sheets, counts, closed, winding, x, w, charge);
    if (order == 1)
        return orc_deposit_linear(nx, L, n_sheets, counts, closed, winding, x, w, charge);
    if (order == 2 || order == 3) {
        long n = 0;
        for (int s = 0; s < n_sheets; ++s)
            n += counts[s];
        return orc_deposit_pic(nx, L, n, x, w, order, charge);
    }
    return orc_deposit(nx, L, n_sheets, counts, closed, winding, x, w, charge);
}

/*
 * Moments of the particles on the mesh: number density n and current density
 * j, by zero-order or first-order weighting of the box particles (Sec. 2.3
 * and Sec. 2.4).
 *
 * Particle s between tracers i and i+1 carries charge q_s = (w_i + w_{i+1})/2
 * spread uniformly over its extent (density q_s / |x_{i+1} - x_i|).
 *   weighting 0 (Eq. rho_sum, Eq. j_sum): cell j gets n_j = sum_s q_s o_js / dx
 *     and j_j = sum_s q_s v~_s o_js / dx, o_js the overlap fraction of
 *     Eq. overlap and v~_s = (m_i v_i + m_{i+1} v_{i+1}) / (m_i + m_{i+1}) the
 *     particle velocity of Sec. 2.3 (masses m = w / qm, so the weights);
 *   weighting 1 (Sec. 2.4): node X_j = j dx gets
 *     n_j = sum_s (1/dx) int q_s b_s(x) W1(x - X_j) dx,
 *     j_j = sum_s (1/dx) int q_s v_s(x) b_s(x) W1(x - X_j) dx,
 *     W1 the hat of half-width dx and v_s(x) the velocity interpolated
 *     linearly along the particle from v_i at x_i to v_{i+1} at x_{i+1}.
 * A zero-length particle is a point charge (first order: the hat weights of
 * its point; velocity v~_s).  Every periodic image counts.  n and j each
 * have nx entries.
 */
static void moments_segment(double xa, double va, double xb, double vb, double q,
                            double vbar, int weighting, int nx, double dx,
                            double *n, double *j)
{
    double a = xa < xb ? xa : xb;
    double b = xa < xb ? xb : xa;
    long ma = (long)floor(a / dx);
    long mb = (long)floor(b / dx);
    if (b == a) {
        if (weighting == 0) {
            int c = wrap_cell(ma, nx);
            n[c] += q / dx;
            j[c] += q * vbar / dx;
        } else {
            double f = a / dx - (double)ma;
            int c0 = wrap_cell(ma, nx), c1 = wrap_cell(ma + 1, nx);
            n[c0] += q * (1.0 - f) / dx;
            n[c1] += q * f / dx;
            j[c0] += q * vbar * (1.0 - f) / dx;
            j[c1] += q * vbar * f / dx;
        }
        return;
    }
    double len = xb - xa;            /* signed: the velocity runs from xa to xb */
    double rho0 = q / fabs(len);
    for (long m = ma - 1; m <= mb + 1; ++m) {
        double lo = a > m * dx ? a : m * dx;
        double hi = b < (m + 1) * dx ? b : (m + 1) * dx;
        if (!(hi > lo))
            continue;
        int c0 = wrap_cell(m, nx), c1 = wrap_cell(m + 1, nx);
        if (weighting == 0) {
            n[c0] += rho0 * (hi - lo) / dx;
            j[c0] += rho0 * vbar * (hi - lo) / dx;
            continue;
        }
        /* s = (x - X_m) / dx in [0, 1): node m weighs 1 - s, node m+1 weighs s */
        double s0 = lo / dx - (double)m, s1 = hi / dx - (double)m;
        double I0 = (s1 - s0) * dx;                       /* int 1 dx         */
        double I1 = 0.5 * (s1 * s1 - s0 * s0) * dx;       /* int s dx         */
        double I2 = (s1 * s1 * s1 - s0 * s0 * s0) / 3.0 * dx; /* int s^2 dx  */
        /* v(x) = va + (vb - va) (x - xa) / len = p + r s on this cell */
        double r = (vb - va) * dx / len;
        double p = va + (vb - va) * ((double)m * dx - xa) / len;
        n[c0] += rho0 * (I0 - I1) / dx;
        n[c1] += rho0 * I1 / dx;
        j[c0] += rho0 * (p * (I0 - I1) + r * (I1 - I2)) / dx;
        j[c1] += rho0 * (p * I1 + r * I2) / dx;
    }
}

int orc_moments(int nx, double L, int n_sheets, const int32_t *counts,
                const uint8_t *closed, const int32_t *winding, const double *x,
                const double *v, const double *w, int weighting, double *n,
                double *j)
{
    double dx = L / nx;
    memset(n, 0, sizeof(double) * (size_t)nx);
    memset(j, 0, sizeof(double) * (size_t)nx);
    long base = 0;
    for (int s = 0; s < n_sheets; ++s) {
        long cnt = counts[s];
        if (cnt < 2)
            return -1;
        long np = closed[s] ? cnt : cnt - 1;
        for (long k = 0; k < np; ++k) {
            long i = base + k, i1 = k + 1 < cnt ? base + k + 1 : base;
            double xb = x[i1] + (k + 1 < cnt ? 0.0 : (double)winding[s] * L);
            double q = 0.5 * (w[i] + w[i1]);
            double vbar = (w[i] * v[i] + w[i1] * v[i1]) / (w[i] + w[i1]);
            moments_segment(x[i], v[i], xb, v[i1], q, vbar, weighting, nx, dx, n, j);
        }
        base += cnt;
    }
    return 0;
}

/*
 * Field solve (Sec. 2.1 with C = 1): n_j = charge_j / dx, rho_j = n_j - mean(n),
 * dE/dx = rho integrated exactly across each cell: E'_0 = 0,
 * E'_{j+1} = E'_j + dx rho_j; E_j = E'_j - mean(E').  rho and E may be NULL.
 */
void orc_field(int nx, double L, const double *charge, double *rho, double *E)
{
    double dx = L / nx;
    double *n = (double *)malloc(sizeof(double) * (size_t)nx);
    double *r = (double *)malloc(sizeof(double) * (size_t)nx);
    double *e = (double *)malloc(sizeof(double) * (size_t)nx);
    double nbar = 0.0;
    for (int j = 0; j < nx; ++j) {
        n[j] = charge[j] / dx;
        nbar += n[j];
    }
    nbar /= nx;
    for (int j = 0; j < nx; ++j)
        r[j] = n[j] - nbar;
    e[0] = 0.0;
    for (int j = 0; j + 1 < nx; ++j)
        e[j + 1] = e[j] + dx * r[j];
    double emean = 0.0;
    for (int j = 0; j < nx; ++j)
        emean += e[j];
    emean /= nx;
    for (int j = 0; j < nx; ++j) {
        if (rho)
            rho[j] = r[j];
        if (E)
            E[j] = e[j] - emean;
    }
    free(n);
    free(r);
    free(e);
}

/*
 * First-order weighting of the box particles (Sec. 2.4): node X_j = j dx gets
 * the charge sum_s q_s int b_s(x) W1(x - X_j) dx, each slice of a particle
 * shared between the two nodes around it by the hat W1 of half-width dx.  This
 * is the first-order density of orc_moments times dx (computed there, with
 * the velocities unused).
 */
int orc_deposit_first(int nx, double L, int n_sheets, const int32_t *counts,
                      const uint8_t *closed, const int32_t *winding,
                      const double *x, const double *w, double *charge)
{
    long n = 0;
    for (int s = 0; s < n_sheets; ++s)
        n += counts[s];
    double *v0 = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    double *j = (double *)malloc(sizeof(double) * (size_t)nx);
    int rc = orc_moments(nx, L, n_sheets, counts, closed, winding, x, v0, w, 1, charge, j);
    double dx = L / nx;
    for (int k = 0; k < nx; ++k)
        charge[k] *= dx;
    free(v0);
    free(j);
    return rc;
}

/*
 * Field solve for charge on the nodes (first-order weighting, Sec. 2.4, with
 * Sec. 2.1, C = 1): n_j = charge_j / dx, rho_j = n_j - mean(n) at X_j, and
 * dE/dx = rho integrated from node to node by the trapezoid rule,
 * E'_0 = 0, E'_{j+1} = E'_j + dx (rho_j + rho_{j+1}) / 2 (rho_nx = rho_0);
 * E_j = E'_j - mean(E').  rho and E may be NULL.
 */
void orc_field_nodes(int nx, double L, const double *charge, double *rho, double *E)
{
    double dx = L / nx;
    double *r = (double *)malloc(sizeof(double) * (size_t)nx);
    double *e = (double *)malloc(sizeof(double) * (size_t)nx);
    double nbar = 0.0;
    for (int j = 0; j < nx; ++j)
        nbar += charge[j] / dx;
    nbar /= nx;
    for (int j = 0; j < nx; ++j)
        r[j] = charge[j] / dx - nbar;
    e[0] = 0.0;
    for (int j = 0; j + 1 < nx; ++j)
        e[j + 1] = e[j] + dx * 0.5 * (r[j] + r[j + 1]);
    double emean = 0.0;
    for (int j = 0; j < nx; ++j)
        emean += e[j];
    emean /= nx;
    for (int j = 0; j < nx; ++j) {
        if (rho)
            rho[j] = r[j];
        if (E)
            E[j] = e[j] - emean;
    }
    free(r);
    free(e);
}

/* Linear-weighting gather of the node field at one position (Sec. 2.3). */
static double gather_one(int nx, double dx, const double *E, double x)
{
    double u = x / dx;
    double m = floor(u);
    double f = u - m;
    int j = wrap_cell((long)m, nx);
    int j1 = j + 1 == nx ? 0 : j + 1;
    return (1.0 - f) * E[j] + f * E[j1];
}

void orc_gather(int nx, double L, const double *E, long n, const double *x,
                double *ex)
{
    double dx = L / nx;
    for (long i = 0; i < n; ++i)
        ex[i] = gather_one(nx, dx, E, x[i]);
}

/* Field energy W_E = 1/2 * integral of E^2 over the box, on the nodes. */
double orc_field_energy(int nx, double L, const double *E)
{
    double dx = L / nx;
    double s = 0.0;
    for (int j = 0; j < nx; ++j)
        s += E[j] * E[j];
    return 0.5 * dx * s;
}

/*
 * Leapfrog run of n_steps SIC steps (solve, gather, move of Sec. 2.3; only
 * the scatter differs from PIC).
 *
 * On entry x, v hold x^0 and v^0 (or v^{-1/2} when half_step_init is 0).
 * With half_step_init != 0 the velocities are first moved back half a step,
 * v^{-1/2} = v^0 - dt/2 qm E^0(x^0).  Step n kicks with E^n at x^n, drifts,
 * then deposits and solves for E^{n+1}.
 *
 * hist (n_steps+1 rows of 4 doubles, may be NULL) gets for every step n:
 *   [W_E^n, KE^n, P^n, total charge]
 * with KE^n = 1/2 sum m (v_{n-1/2}^2 + v_{n+1/2}^2)/2 and
 * P^n = sum m (v_{n-1/2} + v_{n+1/2})/2 (time-centred on step n), mass
 * m_i = w_i / qm.  Row n_steps has W_E of the final field and NaN for KE, P.
 * e_hist (n_steps+1 rows of nx, may be NULL) gets every E^n.
 * On exit x = x^{n_steps}, v = v^{n_steps-1/2}, E_out = E^{n_steps} (may be NULL).
 * order selects the deposit: 0 box particles (Sec. 2.3), 1 piecewise linear
 * (Sec. 2.5), 2 PIC nearest grid point, 3 PIC cloud in cell (Sec. 2.4),
 * 4 first-order weighting of the box particles onto the nodes (Sec. 2.4),
 * whose field comes from orc_field_nodes.
 */
int orc_run(int nx, double L, double dt, double qm, int half_step_init,
            int n_sheets, const int32_t *counts, const uint8_t *closed,
            const int32_t *winding, long n_tracers, double *x, double *v,
            const double *w, int n_steps, double *hist, double *e_hist,
            double *E_out, int order)
{
    double *charge = (double *)malloc(sizeof(double) * (size_t)nx);
    double *E = (double *)malloc(sizeof(double) * (size_t)nx);
    double *ex = (double *)malloc(sizeof(double) * (size_t)n_tracers);
    int rc = deposit_order(order, nx, L, n_sheets, counts, closed, winding, x, w, charge);
    if (rc)
        goto done;
    if (order == 4)
        orc_field_nodes(nx, L, charge, NULL, E);
    else
        orc_field(nx, L, charge, NULL, E);
    if (half_step_init) {
        orc_gather(nx, L, E, n_tracers, x, ex);
        for (long i = 0; i < n_tracers; ++i)
            v[i] -= 0.5 * dt * qm * ex[i];
    }
    for (int step = 0; step <= n_steps; ++step) {
        double qtot = 0.0;
        for (int j = 0; j < nx; ++j)
            qtot += charge[j];
        if (e_hist)
            memcpy(e_hist + (size_t)step * nx, E, sizeof(double) * (size_t)nx);
        double we = orc_field_energy(nx, L, E);
        if (step == n_steps) {
            if (hist) {
                double *h = hist + 4 * (size_t)step;
                h[0] = we;
                h[1] = NAN;
                h[2] = NAN;
                h[3] = qtot;
            }
            break;
        }
        orc_gather(nx, L, E, n_tracers, x, ex);
        double ke = 0.0, p = 0.0;
        for (long i = 0; i < n_tracers; ++i) {
            double m = w[i] / qm;
            double vold = v[i];
            double vnew = vold + dt * qm * ex[i];
            ke += 0.5 * m * 0.5 * (vold * vold + vnew * vnew);
            p += m * 0.5 * (vold + vnew);
            v[i] = vnew;
            x[i] += dt * vnew;
        }
        if (hist) {
            double *h = hist + 4 * (size_t)step;
            h[0] = we;
            h[1] = ke;
            h[2] = p;
            h[3] = qtot;
        }
        rc = deposit_order(order, nx, L, n_sheets, counts, closed, winding, x, w, charge);
        if (rc)
            goto done;
        if (order == 4)
            orc_field_nodes(nx, L, charge, NULL, E);
        else
            orc_field(nx, L, charge, NULL, E);
    }
    if (E_out)
        memcpy(E_out, E, sizeof(double) * (size_t)nx);
done:
    free(charge);
    free(E);
    free(ex);
    return rc;
}

/*
 * One pass of the refinement of Sec. 2.6 over all sheets, in place: every
 * particle longer than l_ref gets a new tracer at its centre, with the mean of
 * its two tracers' velocities, and each half carries half the particle's
 * charge.  x, v, qseg hold the n tracers of the sheets (counts[], updated)
 * with room for cap; qseg[i] is the charge of the particle starting at tracer
 * i (see orc_deposit_seg).  Returns the number of new tracers, or -1 when they
 * do not fit in cap.
 */
long orc_refine(double L, int n_sheets, int32_t *counts, const uint8_t *closed,
                const int32_t *winding, long cap, double *x, double *v,
                double *qseg, double l_ref)
{
    long n = 0, added = 0;
    for (int s = 0; s < n_sheets; ++s)
        n += counts[s];
    /* count first, so nothing moves when the result would not fit */
    long base = 0;
    for (int s = 0; s < n_sheets; ++s) {
        long c = counts[s];
        long np = closed[s] ? c : c - 1;
        for (long k = 0; k < np; ++k) {
            double xb = k + 1 < c ? x[base + k + 1] : x[base] + (double)winding[s] * L;
            if (fabs(xb - x[base + k]) > l_ref)
                ++added;
        }
        base += c;
    }
    if (added == 0)
        return 0;
    if (n + added > cap)
        return -1;
    /* build the refined sheets back to front so no tracer is overwritten
       before it is read */
    long src_end = n, dst_end = n + added;
    for (int s = n_sheets - 1; s >= 0; --s) {
        long c = counts[s];
        long b = src_end - c;
        long grow = 0;
        long np = closed[s] ? c : c - 1;
        for (long k = 0; k < np; ++k) {
            double xb = k + 1 < c ? x[b + k + 1] : x[b] + (double)winding[s] * L;
            if (fabs(xb - x[b + k]) > l_ref)
                ++grow;
        }
        long d = dst_end;
        for (long k = c - 1; k >= 0; --k) {
            int split = 0;
            double xb = 0.0, vb = 0.0;
            if (k < np) {
                xb = k + 1 < c ? x[b + k + 1] : x[b] + (double)winding[s] * L;
                vb = k + 1 < c ? v[b + k + 1] : v[b];
                split = fabs(xb - x[b + k]) > l_ref;
            }
            double xk = x[b + k], vk = v[b + k], qk = qseg[b + k];
            if (split) {
                --d;
                x[d] = 0.5 * (xk + xb);
                v[d] = 0.5 * (vk + vb);
                qseg[d] = 0.5 * qk;
                --d;
                x[d] = xk;
                v[d] = vk;
                qseg[d] = 0.5 * qk;
            } else {
                --d;
                x[d] = xk;
                v[d] = vk;
                qseg[d] = qk;
            }
        }
        counts[s] = (int32_t)(c + grow);
        src_end = b;
        dst_end = d;
    }
    return added;
}

/* The longest particle of the sheets. */
static double longest_particle(double L, int n_sheets, const int32_t *counts,
                               const uint8_t *closed, const int32_t *winding,
                               const double *x)
{
    double m = 0.0;
    long base = 0;
    for (int s = 0; s < n_sheets; ++s) {
        long c = counts[s];
        long np = closed[s] ? c : c - 1;
        for (long k = 0; k < np; ++k) {
            double xb = k + 1 < c ? x[base + k + 1] : x[base] + (double)winding[s] * L;
            double len = fabs(xb - x[base + k]);
            if (len > m)
                m = len;
        }
        base += c;
    }
    return m;
}

/*
 * Leapfrog run of box particles with per-particle charges (qseg, as for
 * orc_deposit_seg), refined after every step in which a particle is longer
 * than l_ref (Sec. 2.6: "if at any time any segment becomes larger than the
 * maximum length, a new tracer is inserted"): orc_refine passes at l_split
 * (0 < l_split <= l_ref) until a pass adds nothing.  l_ref <= 0 or infinite
 * never refines.  Velocities are v^{-1/2} on entry.  Each step: field of the
 * current charge, W[step] = its field energy, kick, drift, refinement when
 * due, deposit of the new tracers.  x, v, qseg have room for cap tracers;
 * counts[] is updated.  n_out (may be NULL) gets the tracer count after every
 * step.  Returns 0, or -1 when the tracers outgrow cap.
 */
int orc_run_refined(int nx, double L, double dt, double qm, int n_sheets,
                    int32_t *counts, const uint8_t *closed, const int32_t *winding,
                    long cap, double *x, double *v, double *qseg, int n_steps,
                    double l_ref, double l_split, double *W, long *n_out)
{
    double *charge = (double *)malloc(sizeof(double) * (size_t)nx);
    double *E = (double *)malloc(sizeof(double) * (size_t)nx);
    int rc = 0;
    long n = 0;
    for (int s = 0; s < n_sheets; ++s)
        n += counts[s];
    double *ex = (double *)malloc(sizeof(double) * (size_t)cap);
    orc_deposit_seg(nx, L, n_sheets, counts, closed, winding, x, qseg, charge);
    for (int step = 0; step < n_steps; ++step) {
        orc_field(nx, L, charge, NULL, E);
        if (W)
            W[step] = orc_field_energy(nx, L, E);
        orc_gather(nx, L, E, n, x, ex);
        for (long i = 0; i < n; ++i) {
            v[i] += dt * qm * ex[i];
            x[i] += dt * v[i];
        }
        if (l_ref > 0.0 && isfinite(l_ref) &&
            longest_particle(L, n_sheets, counts, closed, winding, x) > l_ref) {
            long added;
            do {
                added = orc_refine(L, n_sheets, counts, closed, winding, cap, x, v, qseg, l_split);
                if (added > 0)
                    n += added;
            } while (added > 0);
            if (added < 0) {
                rc = -1;
                break;
            }
        }
        if (n_out)
            n_out[step] = n;
        orc_deposit_seg(nx, L, n_sheets, counts, closed, winding, x, qseg, charge);
    }
    free(charge);
    free(E);
    free(ex);
    return rc;
}
