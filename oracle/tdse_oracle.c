/*
 * tdse_oracle.c -- plain FP64 CPU reference of the FDTD leapfrog for the 3-D
 * time-dependent Schrodinger equation (Nagaya, Omatsu, Packwood, arXiv 2401.07416).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA library is
 * checked against.  It shares no code, header, table or helper with the CUDA
 * library, and only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark may load it.  It is written for a reader checking it against the
 * paper, not for speed: the update is Eqs. 8-9 term by term, neighbours follow
 * Eqs. 13-14 (wrap with mod) or a zero wall, and every sum is FP64.
 *
 * Layout: arrays are [nz][ny][nx], x fastest, unpadded.
 * Units: atomic units are not assumed; hbar and mass are parameters.
 *
 * Readings of points where the paper is silent (each is also listed in the
 * design notes of the repository):
 *   - I at t = -dt/2 is Im psi0 - (1/2) A[Re psi0] (a second-order backward
 *     half step; the paper gives psi at t = 0 only, Sec. 2.1 after Eq. 9);
 *   - the absorbing layer is a per-plane factor M_k = cos^2(eta*(pi/2)*d/W),
 *     d = 1..W the depth into a W-cell layer at either z end, applied to both
 *     parts after each full step (replaces the CAP of Eq. 10);
 *   - the detector records the probability flux through the face between
 *     planes kd and kd+1, j = hbar/(m hz) * (R_kd I_kd+1 - R_kd+1 I_kd), with R at
 *     step n and I at n+1/2 before the mask (Eq. 15 records the density on a
 *     plane instead);
 *   - the potential of an atom is -Z phi(r): phi = 1/rho (rho = sqrt(r^2 + a^2))
 *     minus its second-order Taylor polynomial in r^2 about the cut-off r_c, for
 *     r < r_c, and 0 beyond (twice differentiable at r_c); distances by minimum
 *     image in periodic axes; r_c <= 0 means phi = 1/rho (no cut-off).
 */
#include <math.h>
#include <omp.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>

/* Thread count of the OpenMP loops below, for timing the oracle serially or on all
 * cores.  The per-node loops give the same results at any count; only the summation
 * order of the atom-gradient reduction depends on it. */
void orc_set_threads(int n) { omp_set_num_threads(n > 0 ? n : 1); }
int orc_max_threads(void) { return omp_get_max_threads(); }

typedef struct {
    int nx, ny, nz;
    double hx, hy, hz, dt, hbar, mass;
    int bc[3];          /* per axis: 0 periodic (Eqs. 13-14), 1 zero wall */
    int mask_lo, mask_hi;
    double mask_eta;
    int det_k;          /* detector face kd (between planes kd and kd+1), -1 off */
    int mask_kind;      /* 0: cos^2 layers; 1: Eq. 10 quadratic absorbing potential, split */
} orc_grid;

static size_t ncells(const orc_grid *g) { return (size_t)g->nx * g->ny * g->nz; }

/* Neumaier's compensated sum: sums over millions of nodes must stay accurate far
 * below the 1e-11 parity bound, which a plain running sum (error up to N eps / 2)
 * does not. */
typedef struct {
    double s, c;
} csum;

static void cadd(csum *a, double x)
{
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x))
        a->c += (a->s - t) + x;
    else
        a->c += (x - t) + a->s;
    a->s = t;
}

static double cval(const csum *a) { return a->s + a->c; }

static size_t at3(const orc_grid *g, int i, int j, int k)
{
    return ((size_t)k * g->ny + j) * g->nx + i;
}

/* Coefficients of Eqs. 8-9: c_a = hbar dt / (2 m h_a^2), c_v = dt / hbar. */
void orc_coefficients(const orc_grid *g, double c[4])
{
    c[0] = g->hbar * g->dt / (2.0 * g->mass * g->hx * g->hx);
    c[1] = g->hbar * g->dt / (2.0 * g->mass * g->hy * g->hy);
    c[2] = g->hbar * g->dt / (2.0 * g->mass * g->hz * g->hz);
    c[3] = g->dt / g->hbar;
}

/* Eq. 11: dt = m / (5 hbar) * min(hx, hy, hz)^2. */
double orc_default_dt(double hx, double hy, double hz, double hbar, double mass)
{
    double h = hx;
    if (hy < h) h = hy;
    if (hz < h) h = hz;
    return mass / (5.0 * hbar) * h * h;
}

/* Eq. 4: lambda = sqrt(2 hbar^2 pi^2 / (m E)). */
double orc_wavelength(double energy, double hbar, double mass)
{
    return sqrt(2.0 * hbar * hbar * M_PI * M_PI / (mass * energy));
}

/* Neighbour index along one axis: Eqs. 13-14 replace i+-1 by (i+-1) mod N on a
 * periodic axis; on a walled axis the value outside [0, N) is zero, signalled
 * here by -1. */
static int nb(int i, int n, int periodic)
{
    if (i >= 0 && i < n) return i;
    if (!periodic) return -1;
    return (i % n + n) % n;
}

static double value_at(const orc_grid *g, const double *f, int i, int j, int k)
{
    int ii = nb(i, g->nx, g->bc[0] == 0);
    int jj = nb(j, g->ny, g->bc[1] == 0);
    int kk = nb(k, g->nz, g->bc[2] == 0);
    if (ii < 0 || jj < 0 || kk < 0) return 0.0;
    return f[at3(g, ii, jj, kk)];
}

/* The bracketed right-hand side shared by Eqs. 8 and 9, applied to field f at
 * node (i, j, k):
 *   c_x (f(i+1) - 2 f(i) + f(i-1)) + c_y (...) + c_z (...) - c_v V f(i).
 * Eq. 9 adds it to psi_I; Eq. 8 subtracts it (applied to psi_I) from psi_R. */
static double rhs(const orc_grid *g, const double c[4], const double *V,
                  const double *f, int i, int j, int k)
{
    double f0 = f[at3(g, i, j, k)];
    double lx = value_at(g, f, i + 1, j, k) - 2.0 * f0 + value_at(g, f, i - 1, j, k);
    double ly = value_at(g, f, i, j + 1, k) - 2.0 * f0 + value_at(g, f, i, j - 1, k);
    double lz = value_at(g, f, i, j, k + 1) - 2.0 * f0 + value_at(g, f, i, j, k - 1);
    double v = V ? V[at3(g, i, j, k)] : 0.0;
    return c[0] * lx + c[1] * ly + c[2] * lz - c[3] * v * f0;
}

/* out = A f for every node, where A is the operator of rhs() (A = -(dt/hbar) H). */
void orc_apply_A(const orc_grid *g, const double *V, const double *f, double *out)
{
    double c[4];
    orc_coefficients(g, c);
#pragma omp parallel for schedule(static)
    for (int k = 0; k < g->nz; ++k)
        for (int j = 0; j < g->ny; ++j)
            for (int i = 0; i < g->nx; ++i)
                out[at3(g, i, j, k)] = rhs(g, c, V, f, i, j, k);
}

/* Absorbing layer factor per z plane (reading: cos^2 profile, see header). */
/* Absorbing factor of one layer plane at depth d = 1..W from the layer's inner
 * edge (d = W is the outermost plane).
 * kind 0: M = cos^2(eta (pi/2) d / W).
 * kind 1: Eq. 10's absorbing potential -i W(d) with the quadratic profile
 *   W(d) = eta (d / W)^2 (eta: the strength at the outermost plane, in energy
 *   units; Eq. 10 grows as the square of the distance into the layer), applied by
 *   operator splitting: the term alone, d psi / dt = -W psi / hbar, advances psi by
 *   exactly exp(-W dt / hbar) over one step. */
static double layer_factor(const orc_grid *g, int d, int W)
{
    if (g->mask_kind == 1) {
        double u = (double)d / W;
        return exp(-g->mask_eta * u * u * g->dt / g->hbar);
    }
    double s = cos(g->mask_eta * 0.5 * M_PI * (double)d / W);
    return s * s;
}

void orc_mask(const orc_grid *g, double *M)
{
    for (int k = 0; k < g->nz; ++k) {
        double m = 1.0;
        if (g->mask_lo > 0 && k < g->mask_lo) m = layer_factor(g, g->mask_lo - k, g->mask_lo);
        if (g->mask_hi > 0 && k >= g->nz - g->mask_hi)
            m = layer_factor(g, k - (g->nz - g->mask_hi) + 1, g->mask_hi);
        M[k] = m;
    }
}

/* Shortest periodic image of a displacement along an axis of period L. */
static double min_image(double d, double L, int periodic)
{
    if (!periodic) return d;
    return d - L * floor(d / L + 0.5);
}

/* Radial profile phi of one softened-Coulomb atom as a function of u = r^2
 * (reading, see header) and its derivative d phi / d u.  With f(u) = (u + a^2)^-1/2
 * and u_c = r_c^2, phi = f(u) - [f(u_c) + f'(u_c)(u - u_c) + f''(u_c)(u - u_c)^2 / 2]
 * for u < u_c, 0 beyond: phi and its first two derivatives vanish at r_c. */
static void profile(double r2, double a2, double rc, double *phi, double *dphi_dr2)
{
    double rho = sqrt(r2 + a2);
    if (rc <= 0.0) {
        *phi = 1.0 / rho;
        *dphi_dr2 = -0.5 / (rho * rho * rho);
        return;
    }
    if (r2 >= rc * rc) {
        *phi = 0.0;
        *dphi_dr2 = 0.0;
        return;
    }
    double rhoc = sqrt(rc * rc + a2);
    double rhoc3 = rhoc * rhoc * rhoc;
    double rhoc5 = rhoc3 * rhoc * rhoc;
    double du = r2 - rc * rc;
    *phi = 1.0 / rho - (1.0 / rhoc - 0.5 * du / rhoc3 + 0.375 * du * du / rhoc5);
    *dphi_dr2 = -0.5 / (rho * rho * rho) - (-0.5 / rhoc3 + 0.75 * du / rhoc5);
}

/* V(r) = sum over atoms of -Z phi(|r - r_a|) at the nodes r = origin + (i hx, j hy, k hz)
 * of grid g, with minimum-image distances along every axis whose period[a] is
 * positive (period[a] <= 0: no periodic images).  atoms: [n][4] rows (x, y, z, Z).
 * With origin 0 and period n h on the periodic axes of g this is the potential of
 * the whole grid; other values evaluate a window of a larger grid. */
void orc_potential_atoms_at(const orc_grid *g, const double origin[3], const double period[3],
                            int n, const double *atoms, double a2, double rc, double *V)
{
#pragma omp parallel for schedule(static)
    for (int k = 0; k < g->nz; ++k)
        for (int j = 0; j < g->ny; ++j)
            for (int i = 0; i < g->nx; ++i) {
                double r[3] = {origin[0] + i * g->hx, origin[1] + j * g->hy, origin[2] + k * g->hz};
                double v = 0.0;
                for (int a = 0; a < n; ++a) {
                    double r2 = 0.0;
                    for (int ax = 0; ax < 3; ++ax) {
                        double d = min_image(r[ax] - atoms[4 * a + ax], period[ax], period[ax] > 0.0);
                        r2 += d * d;
                    }
                    double phi, dphi;
                    profile(r2, a2, rc, &phi, &dphi);
                    v += -atoms[4 * a + 3] * phi;
                }
                V[at3(g, i, j, k)] = v;
            }
}

void orc_potential_atoms(const orc_grid *g, int n, const double *atoms, double a2, double rc,
                         double *V)
{
    const double origin[3] = {0.0, 0.0, 0.0};
    const double period[3] = {g->bc[0] == 0 ? g->nx * g->hx : 0.0,
                              g->bc[1] == 0 ? g->ny * g->hy : 0.0,
                              g->bc[2] == 0 ? g->nz * g->hz : 0.0};
    orc_potential_atoms_at(g, origin, period, n, atoms, a2, rc, V);
}

/* Chain rule from dL/dV to the atom parameters: out[4a + (0,1,2,3)] =
 * dL/d(x_a, y_a, z_a, Z_a) = sum over nodes of dL/dV * dV/d(param). */
void orc_atom_gradient(const orc_grid *g, int n, const double *atoms, double a2, double rc,
                       const double *dLdV, double *out)
{
    double L[3] = {g->nx * g->hx, g->ny * g->hy, g->nz * g->hz};
    for (int a = 0; a < n; ++a) {
        double gx = 0.0, gy = 0.0, gz = 0.0, gZ = 0.0;
#pragma omp parallel for reduction(+ : gx, gy, gz, gZ) schedule(static)
        for (int k = 0; k < g->nz; ++k)
            for (int j = 0; j < g->ny; ++j)
                for (int i = 0; i < g->nx; ++i) {
                    double r[3] = {i * g->hx, j * g->hy, k * g->hz};
                    double d[3], r2 = 0.0;
                    for (int ax = 0; ax < 3; ++ax) {
                        d[ax] = min_image(r[ax] - atoms[4 * a + ax], L[ax], g->bc[ax] == 0);
                        r2 += d[ax] * d[ax];
                    }
                    double phi, dphi;
                    profile(r2, a2, rc, &phi, &dphi);
                    double w = dLdV[at3(g, i, j, k)];
                    double Z = atoms[4 * a + 3];
                    /* V_a = -Z phi(r^2), d(r^2)/d(x_a) = -2 (x - x_a) */
                    gx += w * (-Z) * dphi * (-2.0 * d[0]);
                    gy += w * (-Z) * dphi * (-2.0 * d[1]);
                    gz += w * (-Z) * dphi * (-2.0 * d[2]);
                    gZ += w * (-phi);
                }
        out[4 * a + 0] = gx;
        out[4 * a + 1] = gy;
        out[4 * a + 2] = gz;
        out[4 * a + 3] = gZ;
    }
}

/* Eq. 3 with a vector wave number: psi0 = prod_a g_a * exp(i k0 . (r - r0)),
 * g_a = exp(-(r_a - r0_a)^2 / (2 sigma_a^2)) (sigma_a <= 0: plane-wave axis,
 * g_a = 1), at the nodes r = origin + (i hx, j hy, k hz), normalised on this grid
 * so that sum |psi0|^2 hx hy hz = 1.  Writes Re psi0 to R and Im psi0 to I. */
void orc_wavepacket_at(const orc_grid *g, const double origin[3], const double r0[3],
                       const double sigma[3], const double k0[3], double *R, double *I)
{
    csum sum = {0.0, 0.0};
    for (int k = 0; k < g->nz; ++k)
        for (int j = 0; j < g->ny; ++j)
            for (int i = 0; i < g->nx; ++i) {
                double r[3] = {origin[0] + i * g->hx, origin[1] + j * g->hy, origin[2] + k * g->hz};
                double amp = 1.0, phase = 0.0;
                for (int ax = 0; ax < 3; ++ax) {
                    double d = r[ax] - r0[ax];
                    if (sigma[ax] > 0.0) amp *= exp(-d * d / (2.0 * sigma[ax] * sigma[ax]));
                    phase += k0[ax] * d;
                }
                size_t c = at3(g, i, j, k);
                R[c] = amp * cos(phase);
                I[c] = amp * sin(phase);
                cadd(&sum, R[c] * R[c] + I[c] * I[c]);
            }
    double s = 1.0 / sqrt(cval(&sum) * g->hx * g->hy * g->hz);
    for (size_t c = 0; c < ncells(g); ++c) {
        R[c] *= s;
        I[c] *= s;
    }
}

void orc_wavepacket(const orc_grid *g, const double r0[3], const double sigma[3],
                    const double k0[3], double *R, double *I)
{
    const double origin[3] = {0.0, 0.0, 0.0};
    orc_wavepacket_at(g, origin, r0, sigma, k0, R, I);
}

/* Staggered start: psi_I lives at half-integer times (Sec. 2.1), so the state
 * needs I at t = -dt/2.  Reading: I(-dt/2) = Im psi0 - (1/2) A[Re psi0], the
 * backward half step of dI/dt = -H R / hbar.  naive != 0 keeps I = Im psi0. */
void orc_init_half(const orc_grid *g, const double *V, const double *R, double *I, int naive)
{
    if (naive) return;
    double *AR = (double *)malloc(ncells(g) * sizeof(double));
    orc_apply_A(g, V, R, AR);
    for (size_t c = 0; c < ncells(g); ++c) I[c] -= 0.5 * AR[c];
    free(AR);
}

/* One leapfrog step n -> n+1 on (R = psi_R^n, I = psi_I^{n-1/2}):
 *   1. Eq. 9: I <- I + rhs(R) at every node (I^{n+1/2});
 *   2. if jmap != NULL: the detector flux j^n at every (x, y) pixel;
 *   3. Eq. 8: R <- R - rhs(I) at every node (R^{n+1});
 *   4. both parts times the absorbing factor of their z plane.
 * Eq. 9 reads only R and Eq. 8 reads only I, so each update is done in place.
 * M may be NULL (no absorbing layer). */
void orc_step(const orc_grid *g, const double *V, const double *M, double *R, double *I,
              double *jmap)
{
    double c[4];
    orc_coefficients(g, c);
#pragma omp parallel for schedule(static)
    for (int k = 0; k < g->nz; ++k)
        for (int j = 0; j < g->ny; ++j)
            for (int i = 0; i < g->nx; ++i)
                I[at3(g, i, j, k)] += rhs(g, c, V, R, i, j, k);
    if (jmap && g->det_k >= 0 && g->det_k + 1 < g->nz) {
        double cj = g->hbar / (g->mass * g->hz);
        int kd = g->det_k;
        for (int j = 0; j < g->ny; ++j)
            for (int i = 0; i < g->nx; ++i)
                jmap[(size_t)j * g->nx + i] =
                    cj * (R[at3(g, i, j, kd)] * I[at3(g, i, j, kd + 1)] -
                          R[at3(g, i, j, kd + 1)] * I[at3(g, i, j, kd)]);
    }
    /* Eq. 8 reads only the new I, so R is updated in place. */
#pragma omp parallel for schedule(static)
    for (int k = 0; k < g->nz; ++k)
        for (int j = 0; j < g->ny; ++j)
            for (int i = 0; i < g->nx; ++i)
                R[at3(g, i, j, k)] -= rhs(g, c, V, I, i, j, k);
    if (M) {
        for (int k = 0; k < g->nz; ++k)
            for (int j = 0; j < g->ny; ++j)
                for (int i = 0; i < g->nx; ++i) {
                    R[at3(g, i, j, k)] *= M[k];
                    I[at3(g, i, j, k)] *= M[k];
                }
    }
}

/* Advance nsteps; accumulates the time-integrated detector flux
 * F += j^n dt into F (if non-NULL) and stores the last j^n into jlast. */
void orc_run(const orc_grid *g, const double *V, int use_mask, double *R, double *I,
             long nsteps, double *F, double *jlast)
{
    double *M = NULL;
    if (use_mask) {
        M = (double *)malloc(g->nz * sizeof(double));
        orc_mask(g, M);
    }
    size_t npix = (size_t)g->nx * g->ny;
    double *j = (F || jlast) ? (double *)calloc(npix, sizeof(double)) : NULL;
    for (long n = 0; n < nsteps; ++n) {
        orc_step(g, V, M, R, I, j);
        if (F)
            for (size_t p = 0; p < npix; ++p) F[p] += j[p] * g->dt;
    }
    if (jlast && j) memcpy(jlast, j, npix * sizeof(double));
    free(j);
    free(M);
}

/* Observables at step n from (R^n, I^{n-1/2}).  The paper defines only the
 * density (Sec. 2.1 after Eq. 9); the others are the scheme's invariants:
 *   out[0] Q = h^3 sum (R R + I^{n+1/2} I^{n-1/2}), conserved by the leapfrog;
 *   out[1] paper norm = h^3 sum (R^2 + I^{n-1/2}^2);
 *   out[2] E = (R.H R + I^{n+1/2}.H I^{n-1/2}) / (R.R + I^{n+1/2}.I^{n-1/2}),
 *          with H = -(hbar/dt) A;
 *   out[3..8] h^3 sum rho * (x, y, z, x^2, y^2, z^2), rho = R R + I^{n+1/2} I^{n-1/2}. */
void orc_observables(const orc_grid *g, const double *V, const double *R, const double *I,
                     double out[9])
{
    size_t n = ncells(g);
    double *AR = (double *)malloc(n * sizeof(double));
    double *AI = (double *)malloc(n * sizeof(double));
    orc_apply_A(g, V, R, AR);
    orc_apply_A(g, V, I, AI);
    csum q = {0, 0}, pn = {0, 0}, e = {0, 0}, mom[6];
    for (int m = 0; m < 6; ++m) mom[m] = (csum){0, 0};
    for (int k = 0; k < g->nz; ++k)
        for (int j = 0; j < g->ny; ++j)
            for (int i = 0; i < g->nx; ++i) {
                size_t c = at3(g, i, j, k);
                double Ip = I[c] + AR[c];
                double rho = R[c] * R[c] + Ip * I[c];
                double x = i * g->hx, y = j * g->hy, z = k * g->hz;
                cadd(&q, rho);
                cadd(&pn, R[c] * R[c] + I[c] * I[c]);
                cadd(&e, -(g->hbar / g->dt) * (R[c] * AR[c] + Ip * AI[c]));
                cadd(&mom[0], rho * x);
                cadd(&mom[1], rho * y);
                cadd(&mom[2], rho * z);
                cadd(&mom[3], rho * x * x);
                cadd(&mom[4], rho * y * y);
                cadd(&mom[5], rho * z * z);
            }
    double h3 = g->hx * g->hy * g->hz;
    out[0] = cval(&q) * h3;
    out[1] = cval(&pn) * h3;
    out[2] = cval(&e) / cval(&q);
    for (int m = 0; m < 6; ++m) out[3 + m] = cval(&mom[m]) * h3;
    free(AR);
    free(AI);
}

/* Reverse-mode gradient of a loss of the time-integrated detector flux
 * F = sum_n j^n dt, by stored states (the plain way: the forward pass keeps
 * every R^n and I^{n+1/2}).
 *
 * Inputs: the initial state (R0 = psi_R^0, I0 = Im psi0 before the half-step
 * start, i.e. what orc_wavepacket writes), V, nsteps, and gF = dL/dF [ny][nx].
 * Output: gV = dL/dV [nz][ny][nx] (includes the dependence of the half-step
 * start on V).  Forward map per step, with A = rhs() and M the mask:
 *   It = I + A R;  j = cj (R_kd It_kd+1 - R_kd+1 It_kd);
 *   Rt = R - A It;  R' = M Rt;  I' = M It.
 * Adjoint (A is symmetric): for n = N-1 .. 0, with (bR, bI) the adjoints of
 * (R^{n+1}, I^{n+1/2}):
 *   bRt = M bR;  bIt = M bI - A bRt + d j/d It;  bR = bRt + A bIt + d j/d R;
 *   bI = bIt;  gV += -c_v (bIt R - bRt It)   (A contains -c_v V f).
 * Finally I^{-1/2} = I0 - A R0 / 2 gives gV += (c_v/2) bI R0. */
void orc_adjoint(const orc_grid *g, const double *V, int use_mask, const double *R0,
                 const double *I0, long nsteps, const double *gF, double *gV)
{
    size_t n = ncells(g);
    double c[4];
    orc_coefficients(g, c);
    double cj = g->hbar / (g->mass * g->hz);
    int kd = g->det_k;
    double *M = (double *)malloc(g->nz * sizeof(double));
    if (use_mask) orc_mask(g, M);
    else for (int k = 0; k < g->nz; ++k) M[k] = 1.0;

    double *Rs = (double *)malloc(n * nsteps * sizeof(double));  /* R^n */
    double *Is = (double *)malloc(n * nsteps * sizeof(double));  /* It^n = I^{n+1/2} before mask */
    double *R = (double *)malloc(n * sizeof(double));
    double *I = (double *)malloc(n * sizeof(double));
    double *tmp = (double *)malloc(n * sizeof(double));
    memcpy(R, R0, n * sizeof(double));
    memcpy(I, I0, n * sizeof(double));
    orc_init_half(g, V, R, I, 0);
    for (long s = 0; s < nsteps; ++s) {
        memcpy(Rs + s * n, R, n * sizeof(double));
        orc_apply_A(g, V, R, tmp);
        for (size_t q = 0; q < n; ++q) I[q] += tmp[q];
        memcpy(Is + s * n, I, n * sizeof(double));
        orc_apply_A(g, V, I, tmp);
        for (size_t q = 0; q < n; ++q) R[q] -= tmp[q];
        for (int k = 0; k < g->nz; ++k)
            for (size_t p = 0; p < (size_t)g->nx * g->ny; ++p) {
                R[(size_t)k * g->nx * g->ny + p] *= M[k];
                I[(size_t)k * g->nx * g->ny + p] *= M[k];
            }
    }

    double *bR = (double *)calloc(n, sizeof(double));
    double *bI = (double *)calloc(n, sizeof(double));
    double *bRt = (double *)malloc(n * sizeof(double));
    double *bIt = (double *)malloc(n * sizeof(double));
    memset(gV, 0, n * sizeof(double));
    size_t plane = (size_t)g->nx * g->ny;
    int flux_on = kd >= 0 && kd + 1 < g->nz;
    for (long s = nsteps - 1; s >= 0; --s) {
        const double *Rn = Rs + s * n;
        const double *It = Is + s * n;
        for (int k = 0; k < g->nz; ++k)
            for (size_t p = 0; p < plane; ++p) {
                bRt[k * plane + p] = M[k] * bR[k * plane + p];
                bIt[k * plane + p] = M[k] * bI[k * plane + p];
            }
        orc_apply_A(g, V, bRt, tmp);
        for (size_t q = 0; q < n; ++q) bIt[q] -= tmp[q];
        if (flux_on)
            for (size_t p = 0; p < plane; ++p) {
                double w = gF[p] * g->dt * cj;
                bIt[(kd + 1) * plane + p] += w * Rn[kd * plane + p];
                bIt[kd * plane + p] -= w * Rn[(kd + 1) * plane + p];
            }
        orc_apply_A(g, V, bIt, tmp);
        for (size_t q = 0; q < n; ++q) bR[q] = bRt[q] + tmp[q];
        if (flux_on)
            for (size_t p = 0; p < plane; ++p) {
                double w = gF[p] * g->dt * cj;
                bR[kd * plane + p] += w * It[(kd + 1) * plane + p];
                bR[(kd + 1) * plane + p] -= w * It[kd * plane + p];
            }
        for (size_t q = 0; q < n; ++q) {
            bI[q] = bIt[q];
            gV[q] += -c[3] * (bIt[q] * Rn[q] - bRt[q] * It[q]);
        }
    }
    for (size_t q = 0; q < n; ++q) gV[q] += 0.5 * c[3] * bI[q] * R0[q];

    free(Rs); free(Is); free(R); free(I); free(tmp);
    free(bR); free(bI); free(bRt); free(bIt); free(M);
}
