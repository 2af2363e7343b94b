/*
 * orc.c -- plain FP64 CPU oracle of the MITHRA FDTD/PIC time step.
 *
 * TEST INFRASTRUCTURE ONLY (see orc.h).  Written from the paper's method
 * chapter as plain loops in the paper's order and notation: no tiling, no
 * sorting, no fusion; particles are summed serially in index order.  The grid
 * loops carry OpenMP pragmas only where every iteration writes its own
 * vertex, so the thread count never changes a result.
 *
 * Readings of the paper that this file takes (the paper is silent, garbled or
 * self-contradictory at these points):
 *   - alpha'_6 = alpha'_7 uses (c dt/dy)^2 in its last term (the printed
 *     second dx is a typo; re-derived from Eq. NSFDtrick).
 *   - source sign: psi^{n+1} gets +(c dt)^2 * mu0 J for A and
 *     +(c dt)^2 * rho/eps0 for phi (the physical sign of Eq. HelmholtzA/F).
 *   - the B_z formula uses A_y in both x-difference terms.
 *   - the CIC weights are w0 = 1 - delta/D, w1 = delta/D (Eq.
 *     fieldInterpolation without the absolute value).
 *   - phi^n belongs to t = (n+1/2) dt and uses rho^{n+1/2} as its source.
 *   - J^{n+1} is deposited at the mid point of the particle's path over the
 *     field step with the CIC weights (Eq. currentIntegral).
 *   - the rest-frame undulator fields follow from the Lorentz transformation
 *     of the lab field: E_x = -gamma0 beta0 c B'_y, B_y = gamma0 B'_y,
 *     B_z = B'_z, at lab position z' = gamma0 (z + beta0 c t).
 *   - the undulator exit (when the length is finite) carries the same taper
 *     as the entrance, in the distance past the exit.
 *   - Mur first order at edges and corners: the one-dimensional condition
 *     along the outward diagonal to the nearest interior vertex, with the
 *     diagonal length as the spacing.
 *   - a particle whose cell leaves [1, n-3] in any axis is lost: it deposits
 *     nothing from that step on.
 */
#include "orc.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* CODATA 2018 (exact SI values for c and e). */
#define ORC_C    299792458.0
#define ORC_E    1.602176634e-19
#define ORC_ME   9.1093837015e-31
#define ORC_EPS0 8.8541878128e-12
#define ORC_MU0  (1.0 / (ORC_EPS0 * ORC_C * ORC_C))
#define ORC_PI   3.14159265358979323846

void orc_constants(double out[5]) {
    out[0] = ORC_C;
    out[1] = ORC_E;
    out[2] = ORC_ME;
    out[3] = ORC_EPS0;
    out[4] = ORC_MU0;
}

static inline int64_t ix(const orc_grid* g, int i, int j, int k) {
    return ((int64_t)k * g->ny + j) * g->nx + i;
}

static inline int64_t ncell(const orc_grid* g) {
    return (int64_t)g->nx * g->ny * g->nz;
}

/* ---------------------------------------------------------------------- */
/* Coefficients: Sec. "Numerical Dispersion in FDTD", Eq. NSFDCoefficient and
 * the alpha' table under Eq. updateEquation.  The standard central-difference
 * scheme is the same table with A = 0. */
int orc_coefficients(const orc_grid* g, double out[6]) {
    double cdt = ORC_C * g->dt;
    double rx2 = (cdt / g->dx) * (cdt / g->dx);
    double ry2 = (cdt / g->dy) * (cdt / g->dy);
    double rz2 = (cdt / g->dz) * (cdt / g->dz);
    double A = 0.0;
    if (g->stencil == 0) {
        double qx = g->dz / g->dx, qy = g->dz / g->dy;
        A = 0.25 * (1.0 + 0.02 / (qx * qx + qy * qy));
    }
    out[0] = A;
    out[1] = 2.0 * (1.0 - (1.0 - 2.0 * A) * rx2 - (1.0 - 2.0 * A) * ry2 - rz2);
    out[2] = rx2;
    out[3] = ry2;
    out[4] = rz2 - 2.0 * A * rx2 - 2.0 * A * ry2;
    out[5] = cdt * cdt;
    /* Stability.  Standard scheme: Eq. CFLcondition.  NSFD: the left side of
     * Eq. NSFDDispersionCD times (c dt)^2 is linear in sin^2(kz dz/2), so its
     * maximum is max(rx2 + ry2, rz2); a real omega needs that <= 1. */
    if (g->stencil == 0) {
        if (rx2 + ry2 >= 1.0) return 1;
        if (rz2 > 1.0 + 1e-12) return 1;
        return 0;
    }
    return (rx2 + ry2 + rz2 < 1.0) ? 0 : 1;
}

/* ---------------------------------------------------------------------- */
/* Potential update, one component: Eq. updateEquation at interior vertices. */
static void update_interior(const orc_grid* g, const double co[6], const double* pm,
                            const double* p, const double* s, double scale, double* pn) {
    const double A = co[0], a1 = co[1], a2 = co[2], a4 = co[3], a6 = co[4], a8 = co[5];
    const int nx = g->nx, ny = g->ny, nz = g->nz;
#pragma omp parallel for schedule(static)
    for (int k = 1; k < nz - 1; ++k) {
        for (int j = 1; j < ny - 1; ++j) {
            for (int i = 1; i < nx - 1; ++i) {
                /* z-weighted neighbour values, Eq. NSFDtrick */
                double bxp = A * p[ix(g, i + 1, j, k - 1)] + (1.0 - 2.0 * A) * p[ix(g, i + 1, j, k)] + A * p[ix(g, i + 1, j, k + 1)];
                double bxm = A * p[ix(g, i - 1, j, k - 1)] + (1.0 - 2.0 * A) * p[ix(g, i - 1, j, k)] + A * p[ix(g, i - 1, j, k + 1)];
                double byp = A * p[ix(g, i, j + 1, k - 1)] + (1.0 - 2.0 * A) * p[ix(g, i, j + 1, k)] + A * p[ix(g, i, j + 1, k + 1)];
                double bym = A * p[ix(g, i, j - 1, k - 1)] + (1.0 - 2.0 * A) * p[ix(g, i, j - 1, k)] + A * p[ix(g, i, j - 1, k + 1)];
                int64_t c = ix(g, i, j, k);
                double v = -pm[c] + a1 * p[c]
                         + a2 * bxp + a2 * bxm
                         + a4 * byp + a4 * bym
                         + a6 * p[ix(g, i, j, k + 1)] + a6 * p[ix(g, i, j, k - 1)];
                if (s) v += a8 * scale * s[c];
                pn[c] = v;
            }
        }
    }
}

static inline int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* First-order Mur condition (Sec. "First Order ABCs"): for a boundary vertex b
 * (every boundary vertex, or with boundary == 2 the edge and corner vertices)
 * with nearest interior vertex q at distance d,
 *   xi_b^{n+1} = beta0 (xi_b^{n-1} + xi_q^{n+1}) + beta1 (xi_b^n + xi_q^n) - xi_q^{n-1}
 * with beta0 = (c dt - d)/(c dt + d), beta1 = 2 d/(c dt + d). */
/* Second-order Mur condition (Sec. "Second Order ABCs") at a face vertex b
 * (exactly one axis on the boundary), written for the face normal to axis a
 * as the paper writes it for z: with q the interior neighbour along a, dn
 * the spacing along a, and t1, t2 the two tangential axes (r_t = c dt / d_t),
 *   xi_b^{n+1} = g0 xi_b^{n-1} + g1 xi_b^n - xi_q^{n-1} + g1 xi_q^n + g0 xi_q^{n+1}
 *              + g5 (xi_q,t1+ + xi_q,t1- + xi_b,t1+ + xi_b,t1-)^n
 *              + g7 (xi_q,t2+ + xi_q,t2- + xi_b,t2+ + xi_b,t2-)^n,
 *   g0 = (c dt - dn)/(c dt + dn),  g1 = dn (2 - r_t1^2 - r_t2^2)/(c dt + dn),
 *   g5 = r_t1^2 dn / (2 (c dt + dn)),  g7 = r_t2^2 dn / (2 (c dt + dn)).
 * These coefficients are those of the Engquist-Majda form with +c/2 in front
 * of the tangential second derivatives (the printed PDE's -c/2 is a sign
 * slip; the printed coefficients follow from +c/2). */
static double mur2_face(const orc_grid* g, const double* pm, const double* p, const double* pn,
                        int i, int j, int k, int qi, int qj, int qk) {
    const double cdt = ORC_C * g->dt;
    const double d[3] = {g->dx, g->dy, g->dz};
    const int a = (qi != i) ? 0 : (qj != j) ? 1 : 2;  /* normal axis */
    const int t1 = (a == 0) ? 1 : 0, t2 = (a == 2) ? 1 : 2;
    const double dn = d[a];
    const double r1 = cdt / d[t1], r2 = cdt / d[t2];
    const double g0 = (cdt - dn) / (cdt + dn);
    const double g1 = dn * (2.0 - r1 * r1 - r2 * r2) / (cdt + dn);
    const double g5 = r1 * r1 * dn / (2.0 * (cdt + dn));
    const double g7 = r2 * r2 * dn / (2.0 * (cdt + dn));
    const int64_t b = ix(g, i, j, k), q = ix(g, qi, qj, qk);
    int e1[3] = {0, 0, 0}, e2[3] = {0, 0, 0};
    e1[t1] = 1;
    e2[t2] = 1;
    double v = g0 * pm[b] + g1 * p[b] - pm[q] + g1 * p[q] + g0 * pn[q];
    v += g5 * (p[ix(g, qi + e1[0], qj + e1[1], qk + e1[2])] + p[ix(g, qi - e1[0], qj - e1[1], qk - e1[2])]
             + p[ix(g, i + e1[0], j + e1[1], k + e1[2])] + p[ix(g, i - e1[0], j - e1[1], k - e1[2])]);
    v += g7 * (p[ix(g, qi + e2[0], qj + e2[1], qk + e2[2])] + p[ix(g, qi - e2[0], qj - e2[1], qk - e2[2])]
             + p[ix(g, i + e2[0], j + e2[1], k + e2[2])] + p[ix(g, i - e2[0], j - e2[1], k - e2[2])]);
    return v;
}

static void mur_boundary(const orc_grid* g, const double* pm, const double* p, double* pn) {
    const int nx = g->nx, ny = g->ny, nz = g->nz;
    const double cdt = ORC_C * g->dt;
    for (int k = 0; k < nz; ++k) {
        for (int j = 0; j < ny; ++j) {
            for (int i = 0; i < nx; ++i) {
                int onb = (i == 0 || i == nx - 1 || j == 0 || j == ny - 1 || k == 0 || k == nz - 1);
                if (!onb) continue;
                int qi = clampi(i, 1, nx - 2), qj = clampi(j, 1, ny - 2), qk = clampi(k, 1, nz - 2);
                int naxes = (qi != i) + (qj != j) + (qk != k);
                if (g->boundary == 2 && naxes == 1) {
                    pn[ix(g, i, j, k)] = mur2_face(g, pm, p, pn, i, j, k, qi, qj, qk);
                    continue;
                }
                double d2 = 0.0;
                if (qi != i) d2 += g->dx * g->dx;
                if (qj != j) d2 += g->dy * g->dy;
                if (qk != k) d2 += g->dz * g->dz;
                double d = sqrt(d2);
                double b0 = (cdt - d) / (cdt + d);
                double b1 = 2.0 * d / (cdt + d);
                int64_t b = ix(g, i, j, k), q = ix(g, qi, qj, qk);
                pn[b] = b0 * (pm[b] + pn[q]) + b1 * (p[b] + p[q]) - pm[q];
            }
        }
    }
}

void orc_potential_step(const orc_grid* g, const double* prev, const double* cur,
                        const double* src, double* next) {
    double co[6];
    orc_coefficients(g, co);
    const int64_t n = ncell(g);
    for (int c = 0; c < 4; ++c) {
        const double* pm = prev + c * n;
        const double* p = cur + c * n;
        const double* s = src + c * n;
        double* pn = next + c * n;
        if (c == 3 && !g->space_charge) {
            memset(pn, 0, sizeof(double) * (size_t)n);
            continue;
        }
        /* source term: mu0 J for A, rho/eps0 for phi */
        double scale = (c < 3) ? ORC_MU0 : 1.0 / ORC_EPS0;
        update_interior(g, co, pm, p, s, scale, pn);
        mur_boundary(g, pm, p, pn);
    }
}

/* ---------------------------------------------------------------------- */
/* E and B at the vertices, Sec. "Field Evaluation". */
void orc_fields(const orc_grid* g, const double* lev_n, const double* lev_np1,
                double* E, double* B) {
    const int64_t n = ncell(g);
    const int nx = g->nx, ny = g->ny, nz = g->nz;
    const double* Axn = lev_n;
    const double* Ayn = lev_n + n;
    const double* Azn = lev_n + 2 * n;
    const double* phn = lev_n + 3 * n;
    const double* Ax1 = lev_np1;
    const double* Ay1 = lev_np1 + n;
    const double* Az1 = lev_np1 + 2 * n;
    const double dx = g->dx, dy = g->dy, dz = g->dz, dt = g->dt;
    memset(E, 0, sizeof(double) * 3 * (size_t)n);
    memset(B, 0, sizeof(double) * 3 * (size_t)n);
#pragma omp parallel for schedule(static)
    for (int k = 1; k < nz - 1; ++k) {
        for (int j = 1; j < ny - 1; ++j) {
            for (int i = 1; i < nx - 1; ++i) {
                int64_t c = ix(g, i, j, k);
                int64_t xp = ix(g, i + 1, j, k), xm = ix(g, i - 1, j, k);
                int64_t yp = ix(g, i, j + 1, k), ym = ix(g, i, j - 1, k);
                int64_t zp = ix(g, i, j, k + 1), zm = ix(g, i, j, k - 1);
                /* B = curl A, averaged over levels n and n+1 */
                double bx0 = (Azn[yp] - Azn[ym]) / (2 * dy) - (Ayn[zp] - Ayn[zm]) / (2 * dz);
                double bx1 = (Az1[yp] - Az1[ym]) / (2 * dy) - (Ay1[zp] - Ay1[zm]) / (2 * dz);
                double by0 = (Axn[zp] - Axn[zm]) / (2 * dz) - (Azn[xp] - Azn[xm]) / (2 * dx);
                double by1 = (Ax1[zp] - Ax1[zm]) / (2 * dz) - (Az1[xp] - Az1[xm]) / (2 * dx);
                double bz0 = (Ayn[xp] - Ayn[xm]) / (2 * dx) - (Axn[yp] - Axn[ym]) / (2 * dy);
                double bz1 = (Ay1[xp] - Ay1[xm]) / (2 * dx) - (Ax1[yp] - Ax1[ym]) / (2 * dy);
                B[c] = 0.5 * (bx0 + bx1);
                B[n + c] = 0.5 * (by0 + by1);
                B[2 * n + c] = 0.5 * (bz0 + bz1);
                /* E = -dA/dt - grad phi, phi^n at (n+1/2) dt */
                E[c] = -(Ax1[c] - Axn[c]) / dt - (phn[xp] - phn[xm]) / (2 * dx);
                E[n + c] = -(Ay1[c] - Ayn[c]) / dt - (phn[yp] - phn[ym]) / (2 * dy);
                E[2 * n + c] = -(Az1[c] - Azn[c]) / dt - (phn[zp] - phn[zm]) / (2 * dz);
            }
        }
    }
}

/* ---------------------------------------------------------------------- */
/* Undulator, Sec. "Undulator Field": lab field of a planar static undulator,
 * B'_y = B0 cosh(ku y) sin(ku zeta), B'_z = B0 sinh(ku y) cos(ku zeta), zeta the
 * lab distance past the entrance; for zeta < 0 the Neumann-shaped fringe
 * B'_y = B0 cosh(ku y) ku zeta exp(-(ku zeta)^2/2), B'_z = B0 sinh(ku y) exp(..).
 * B0 from K = e B0 lambda_u / (2 pi m c).  Transformed to the frame moving with
 * beta0 along +z. */
/* Optical undulator (input group UNDULATOR with undulator-type optical and
 * beam-type plane-wave; the signal types of the FIELD section): in the lab the
 * vector potential is A' = p A0 s(tau) with tau = t' - d (z' - z0)/c, so
 *   E' = -dA'/dt' = -p A0 s'(tau),   B' = curl A' = -(d/c) z x p A0 s'(tau).
 * s is the signal of the paper's list with x = tau - t0, w = 2 pi c / lambda0,
 * carrier C = cos(w x + cep), envelope width tau_v (variance / c):
 *   Gaussian  s = C exp(-2 ln2 x^2/tau_v^2)
 *   sech      s = C / cosh(x/tau_v)
 *   flat-top  s = C exp(-2 ln2 x^2/tau_v^2) for x <= 0, s = C for x > 0
 *   Neumann   s = -4 ln2 (x/tau_v) C exp(-2 ln2 x^2/tau_v^2)
 * (the Neumann signal is written with x/tau_v where the paper prints
 * x/tau^2, so that A0 keeps its meaning as the amplitude).  s' is the exact
 * derivative.  The rest frame moves at +beta0 c along z:
 *   E_perp = gamma0 (E' + v x B'),  B_perp = gamma0 (B' - v x E'/c^2). */
static double signal_derivative(const orc_undulator* u, double x) {
    const double w = 2.0 * ORC_PI * ORC_C / u->lambda_l;
    const double tv = u->variance / ORC_C;
    const double ph = w * x + u->cep;
    const double C = cos(ph), dC = -w * sin(ph);
    const double a = 2.0 * log(2.0) / (tv * tv);
    switch (u->signal) {
        case 0: {
            const double G = exp(-a * x * x);
            const double k = -4.0 * log(2.0) / tv;
            /* d/dx [k x C G] */
            return k * (C * G + x * dC * G + x * C * (-2.0 * a * x) * G);
        }
        case 1: {
            const double G = exp(-a * x * x);
            return dC * G + C * (-2.0 * a * x) * G;
        }
        case 2: {
            const double ch = cosh(x / tv);
            return dC / ch - C * tanh(x / tv) / (tv * ch);
        }
        default: {
            if (x > 0.0) return dC;
            const double G = exp(-a * x * x);
            return dC * G + C * (-2.0 * a * x) * G;
        }
    }
}

/* the signal with an extra carrier phase ph (the Gaussian beam's Gouy phase) */
static double signal_value(const orc_undulator* u, double x, double ph) {
    const double w = 2.0 * ORC_PI * ORC_C / u->lambda_l;
    const double tv = u->variance / ORC_C;
    const double C = cos(w * x + u->cep + ph);
    const double a = 2.0 * log(2.0) / (tv * tv);
    switch (u->signal) {
        case 0: return -4.0 * log(2.0) * (x / tv) * C * exp(-a * x * x);
        case 1: return C * exp(-a * x * x);
        case 2: return C / cosh(x / tv);
        default: return x > 0.0 ? C : C * exp(-a * x * x);
    }
}

static double wave_tau(const orc_undulator* u, double z, double t) {
    const double g0 = u->gamma0;
    const double b0 = sqrt(1.0 - 1.0 / (g0 * g0));
    const double zl = g0 * (z + b0 * ORC_C * t);
    const double tl = g0 * (t + b0 * z / ORC_C);
    return tl - (double)u->direction * (zl - u->z0_lab) / ORC_C;
}

void orc_incident_potential(const orc_undulator* u, double x, double y, double z, double t,
                            double out[2]) {
    const double A0 = u->a0 * ORC_ME * ORC_C / ORC_E;
    const double tau = wave_tau(u, z, t);
    double s;
    if (u->beam == 1) {
        const double g0 = u->gamma0;
        const double b0 = sqrt(1.0 - 1.0 / (g0 * g0));
        const double zl = g0 * (z + b0 * ORC_C * t);
        const double zeta = (double)u->direction * (zl - u->z0_lab);
        const double pn = sqrt(u->pol_x * u->pol_x + u->pol_y * u->pol_y);
        const double px = u->pol_x / pn, py = u->pol_y / pn;
        const double X = x - u->x0_lab, Y = y - u->y0_lab;
        const double off[2] = {px * X + py * Y, -py * X + px * Y};  /* xi, eta */
        const double w0[2] = {u->w_par, u->w_perp};
        double amp = 1.0, delay = 0.0, gouy = 0.0;
        for (int a = 0; a < 2; ++a) {
            const double zr = ORC_PI * w0[a] * w0[a] / u->lambda_l;
            const double w = w0[a] * sqrt(1.0 + (zeta / zr) * (zeta / zr));
            const double invR = zeta / (zeta * zeta + zr * zr);
            amp *= sqrt(w0[a] / w) * exp(-off[a] * off[a] / (w * w));
            delay += off[a] * off[a] * invR / (2.0 * ORC_C);
            gouy += 0.5 * atan(zeta / zr);
        }
        s = amp * signal_value(u, tau - delay - u->offset / ORC_C, gouy);
    } else {
        s = signal_value(u, tau - u->offset / ORC_C, 0.0);
    }
    out[0] = u->pol_x * A0 * s;
    out[1] = u->pol_y * A0 * s;
}

void orc_incident_potential_many(const orc_undulator* u, int64_t n, const double* x,
                                 const double* y, const double* z, const double* t,
                                 double* out) {
    for (int64_t q = 0; q < n; ++q) orc_incident_potential(u, x[q], y[q], z[q], t[q], out + 2 * q);
}

void orc_seed_correction(const orc_grid* g, const orc_undulator* seed, double t_n,
                         double* next) {
    double co[6];
    orc_coefficients(g, co);
    const double A = co[0], a2 = co[2], a4 = co[3], a6 = co[4];
    const int64_t n = ncell(g);
    const int ks = 2, kt = 3;
    const int64_t nxy = (int64_t)g->nx * g->ny;
    /* the incident potential at every vertex of the two planes */
    double* fs = (double*)malloc(sizeof(double) * 2 * nxy);
    double* ft = (double*)malloc(sizeof(double) * 2 * nxy);
    for (int j = 0; j < g->ny; ++j) {
        for (int i = 0; i < g->nx; ++i) {
            const double x = g->x0 + i * g->dx, y = g->y0 + j * g->dy;
            const int64_t v = (int64_t)j * g->nx + i;
            orc_incident_potential(seed, x, y, g->z0 + ks * g->dz, t_n, fs + 2 * v);
            orc_incident_potential(seed, x, y, g->z0 + kt * g->dz, t_n, ft + 2 * v);
        }
    }
#define F(f, i, j, c) (f)[2 * ((int64_t)(j) * g->nx + (i)) + (c)]
    for (int c = 0; c < 2; ++c) {
        double* pn = next + c * n;
        for (int j = 1; j < g->ny - 1; ++j) {
            for (int i = 1; i < g->nx - 1; ++i) {
                /* scattered-field plane: its k+1 neighbours hold the total field */
                pn[ix(g, i, j, ks)] -= A * (a2 * F(ft, i + 1, j, c) + a2 * F(ft, i - 1, j, c)
                                            + a4 * F(ft, i, j + 1, c) + a4 * F(ft, i, j - 1, c))
                                     + a6 * F(ft, i, j, c);
                /* total-field plane: its k-1 neighbours hold the scattered field */
                pn[ix(g, i, j, kt)] += A * (a2 * F(fs, i + 1, j, c) + a2 * F(fs, i - 1, j, c)
                                            + a4 * F(fs, i, j + 1, c) + a4 * F(fs, i, j - 1, c))
                                     + a6 * F(fs, i, j, c);
            }
        }
    }
#undef F
    free(fs);
    free(ft);
}

static void optical_field(const orc_undulator* u, double z, double t, double E[3], double B[3]) {
    const double g0 = u->gamma0;
    const double b0 = sqrt(1.0 - 1.0 / (g0 * g0));
    const double d = (double)u->direction;
    const double zl = g0 * (z + b0 * ORC_C * t);
    const double tl = g0 * (t + b0 * z / ORC_C);
    const double tau = tl - d * (zl - u->z0_lab) / ORC_C;
    const double A0 = u->a0 * ORC_ME * ORC_C / ORC_E;
    const double sp = signal_derivative(u, tau - u->offset / ORC_C);
    /* lab fields: E' = -p A0 s', B' = -(d/c) z x p A0 s' with z x p = (-p_y, p_x, 0) */
    const double Ex = -u->pol_x * A0 * sp, Ey = -u->pol_y * A0 * sp;
    const double Bx = -(d / ORC_C) * (-u->pol_y) * A0 * sp;
    const double By = -(d / ORC_C) * (u->pol_x) * A0 * sp;
    /* v x F = b0 c z x F = b0 c (-F_y, F_x, 0) */
    E[0] = g0 * (Ex - b0 * ORC_C * By);
    E[1] = g0 * (Ey + b0 * ORC_C * Bx);
    E[2] = 0.0;
    B[0] = g0 * (Bx + b0 * Ey / ORC_C);
    B[1] = g0 * (By - b0 * Ex / ORC_C);
    B[2] = 0.0;
}

void orc_undulator_field(const orc_undulator* u, double y, double z, double t,
                         double E[3], double B[3]) {
    if (u->type == 1) {
        optical_field(u, z, t, E, B);
        return;
    }
    const double g0 = u->gamma0;
    const double b0 = sqrt(1.0 - 1.0 / (g0 * g0));
    const double ku = 2.0 * ORC_PI / u->lambda_u;
    const double B0 = 2.0 * ORC_PI * ORC_ME * ORC_C * u->K / (ORC_E * u->lambda_u);
    /* lab position of the rest-frame event (z, t) */
    const double zlab = g0 * (z + b0 * ORC_C * t);
    const double zeta = zlab - u->z_ent_lab;
    const double ch = cosh(ku * y), sh = sinh(ku * y);
    double By_l = 0.0, Bz_l = 0.0;
    if (zeta < 0.0) {
        if (u->fringe) {
            double a = ku * zeta;
            By_l = B0 * ch * a * exp(-0.5 * a * a);
            Bz_l = B0 * sh * exp(-0.5 * a * a);
        }
    } else if (u->length_lab > 0.0 && zeta > u->length_lab) {
        if (u->fringe) {
            double a = ku * (zeta - u->length_lab);
            By_l = B0 * ch * a * exp(-0.5 * a * a);
            Bz_l = B0 * sh * exp(-0.5 * a * a);
        }
    } else {
        By_l = B0 * ch * sin(ku * zeta);
        Bz_l = B0 * sh * cos(ku * zeta);
    }
    /* E' = 0, B' = (0, By_l, Bz_l); frame velocity +beta0 c z:
     * E_perp = gamma0 (v x B'), B_perp = gamma0 B'_perp, B_par = B'_par. */
    E[0] = -g0 * b0 * ORC_C * By_l;
    E[1] = 0.0;
    E[2] = 0.0;
    B[0] = 0.0;
    B[1] = g0 * By_l;
    B[2] = Bz_l;
}

/* ---------------------------------------------------------------------- */
/* Boris scheme, Eq. BorisScheme, written for a general charge-to-mass ratio
 * qm (the paper's -e/m for electrons):
 *   t1 = u + qm dtb E/(2c); alpha = qm dtb / (2 sqrt(1 + t1.t1))
 *   t2 = t1 + alpha t1 x B; t3 = t1 + t2 x (2 alpha B)/(1 + alpha^2 B.B)
 *   u' = t3 + qm dtb E/(2c). */
static void cross(const double a[3], const double b[3], double o[3]) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

void orc_boris(double u[3], const double E[3], const double B[3], double qm, double dtb) {
    double h = qm * dtb / (2.0 * ORC_C);
    double t1[3] = {u[0] + h * E[0], u[1] + h * E[1], u[2] + h * E[2]};
    double alpha = qm * dtb / (2.0 * sqrt(1.0 + t1[0] * t1[0] + t1[1] * t1[1] + t1[2] * t1[2]));
    double c1[3];
    cross(t1, B, c1);
    double t2[3] = {t1[0] + alpha * c1[0], t1[1] + alpha * c1[1], t1[2] + alpha * c1[2]};
    double bb = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
    double f = 2.0 * alpha / (1.0 + alpha * alpha * bb);
    double s[3] = {f * B[0], f * B[1], f * B[2]};
    double c2[3];
    cross(t2, s, c2);
    double t3[3] = {t1[0] + c2[0], t1[1] + c2[1], t1[2] + c2[2]};
    u[0] = t3[0] + h * E[0];
    u[1] = t3[1] + h * E[1];
    u[2] = t3[2] + h * E[2];
}

/* ---------------------------------------------------------------------- */
/* Cell index and offset of a position along one axis (the paper's
 * (i, delta) of Fig. FDTDPICFig1). */
static inline int cell_of(double r, double r0, double d, double* w1) {
    double s = (r - r0) / d;
    double f = floor(s);
    *w1 = s - f;
    return (int)f;
}

static inline int valid_cell(const orc_grid* g, int ci, int cj, int ck) {
    return ci >= 1 && ci <= g->nx - 3 && cj >= 1 && cj <= g->ny - 3 && ck >= 1 && ck <= g->nz - 3;
}

static int locate(const orc_grid* g, double x, double y, double z, int c[3], double w1[3]) {
    c[0] = cell_of(x, g->x0, g->dx, &w1[0]);
    c[1] = cell_of(y, g->y0, g->dy, &w1[1]);
    c[2] = cell_of(z, g->z0, g->dz, &w1[2]);
    return valid_cell(g, c[0], c[1], c[2]);
}

/* Trilinear weights of Eq. fieldInterpolation: w0 = 1 - delta/D, w1 = delta/D. */
static inline double wgt(int I, double w1) { return I ? w1 : 1.0 - w1; }

static void gather(const orc_grid* g, const double* F, const int c[3], const double w1[3],
                   double out[3]) {
    const int64_t n = ncell(g);
    out[0] = out[1] = out[2] = 0.0;
    for (int K = 0; K < 2; ++K)
        for (int J = 0; J < 2; ++J)
            for (int I = 0; I < 2; ++I) {
                double w = wgt(I, w1[0]) * wgt(J, w1[1]) * wgt(K, w1[2]);
                int64_t v = ix(g, c[0] + I, c[1] + J, c[2] + K);
                out[0] += w * F[v];
                out[1] += w * F[n + v];
                out[2] += w * F[2 * n + v];
            }
}

static void scatter(const orc_grid* g, double* F, const int c[3], const double w1[3],
                    double amount) {
    for (int K = 0; K < 2; ++K)
        for (int J = 0; J < 2; ++J)
            for (int I = 0; I < 2; ++I) {
                double w = wgt(I, w1[0]) * wgt(J, w1[1]) * wgt(K, w1[2]);
                F[ix(g, c[0] + I, c[1] + J, c[2] + K)] += w * amount;
            }
}

int64_t orc_mark_lost(const orc_grid* g, int64_t np, const double* x, const double* y,
                      const double* z, int32_t* lost) {
    int64_t nl = 0;
    for (int64_t p = 0; p < np; ++p) {
        int c[3];
        double w1[3];
        if (!locate(g, x[p], y[p], z[p], c, w1)) lost[p] = 1;
        if (lost[p]) ++nl;
    }
    return nl;
}

void orc_deposit_rho(const orc_grid* g, double q_macro, int64_t np, const double* x,
                     const double* y, const double* z, const int32_t* lost, double* rho_out) {
    const double V = g->dx * g->dy * g->dz;
    for (int64_t p = 0; p < np; ++p) {
        if (lost[p]) continue;
        int c[3];
        double w1[3];
        if (!locate(g, x[p], y[p], z[p], c, w1)) continue;
        scatter(g, rho_out, c, w1, q_macro / V);
    }
}

/* Sec. "Update Algorithm" + "Current Deposition": per particle, n_sub Boris
 * steps of dt_b = dt/n_sub with the grid E,B held at t_half and the undulator
 * field at each sub-step time; then J^{n+1} = (q/V) (r_end - r_start)/dt at
 * the mid point and rho^{n+3/2} = q/V at r_end, both with the CIC weights.
 * r_end - r_start is kept as the sum of the sub-step displacements rather than
 * formed by subtracting two absolute positions, which would cancel most of
 * its digits when the displacement is small against the position. */
int64_t orc_push_deposit(const orc_grid* g, const orc_undulator* und, double q_macro,
                         double t_half, const double* E, const double* B,
                         int64_t np, double* x, double* y, double* z,
                         double* ux, double* uy, double* uz, int32_t* lost,
                         double* src_out) {
    const int64_t n = ncell(g);
    const double qm = -ORC_E / ORC_ME; /* electrons */
    const double dtb = g->dt / g->n_sub;
    const double V = g->dx * g->dy * g->dz;
    int64_t newly_lost = 0;
    for (int64_t p = 0; p < np; ++p) {
        if (lost[p]) continue;
        double r0[3] = {x[p], y[p], z[p]};
        double r[3] = {x[p], y[p], z[p]};
        double dr[3] = {0.0, 0.0, 0.0}; /* r^{n+3/2} - r^{n+1/2}, summed per sub-step */
        double u[3] = {ux[p], uy[p], uz[p]};
        int ok = 1;
        for (int m = 0; m < g->n_sub; ++m) {
            int c[3];
            double w1[3];
            if (!locate(g, r[0], r[1], r[2], c, w1)) { ok = 0; break; }
            double Eg[3], Bg[3], Eu[3], Bu[3];
            gather(g, E, c, w1, Eg);
            gather(g, B, c, w1, Bg);
            orc_undulator_field(und, r[1], r[2], t_half + m * dtb, Eu, Bu);
            double Et[3] = {Eg[0] + Eu[0], Eg[1] + Eu[1], Eg[2] + Eu[2]};
            double Bt[3] = {Bg[0] + Bu[0], Bg[1] + Bu[1], Bg[2] + Bu[2]};
            orc_boris(u, Et, Bt, qm, dtb);
            double gam = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
            for (int a = 0; a < 3; ++a) {
                double step = ORC_C * dtb * u[a] / gam;
                r[a] += step;
                dr[a] += step;
            }
        }
        x[p] = r[0]; y[p] = r[1]; z[p] = r[2];
        ux[p] = u[0]; uy[p] = u[1]; uz[p] = u[2];
        int c[3];
        double w1[3];
        if (ok) ok = locate(g, r[0], r[1], r[2], c, w1);
        if (!ok) {
            lost[p] = 1;
            ++newly_lost;
            continue;
        }
        /* rho^{n+3/2} at the end position */
        scatter(g, src_out + 3 * n, c, w1, q_macro / V);
        /* J^{n+1} at the mid point */
        double rm[3] = {r0[0] + 0.5 * dr[0], r0[1] + 0.5 * dr[1], r0[2] + 0.5 * dr[2]};
        int cm[3];
        double wm[3];
        locate(g, rm[0], rm[1], rm[2], cm, wm);
        for (int a = 0; a < 3; ++a) {
            double J = (q_macro / V) * dr[a] / g->dt;
            scatter(g, src_out + a * n, cm, wm, J);
        }
    }
    return newly_lost;
}

/* ---------------------------------------------------------------------- */
/* Total power through the vertex plane k_p, in the lab frame: the grid fields
 * are transformed to the lab (frame velocity beta0 along +z),
 *   E'_x = g0 (E_x + b0 c B_y), E'_y = g0 (E_y - b0 c B_x),
 *   B'_x = g0 (B_x - b0 E_y / c), B'_y = g0 (B_y + b0 E_x / c),
 * and P' = sum over interior (i,j) of (E'_x B'_y - E'_y B'_x)/mu0 dx dy. */
void orc_radiated_power(const orc_grid* g, double gamma0, const double* E, const double* B,
                        int32_t k_p, double t, double* p_lab, double* t_lab, double* z_lab) {
    const int64_t n = ncell(g);
    const double b0 = sqrt(1.0 - 1.0 / (gamma0 * gamma0));
    double sum = 0.0;
    for (int j = 1; j < g->ny - 1; ++j) {
        for (int i = 1; i < g->nx - 1; ++i) {
            int64_t c = ix(g, i, j, k_p);
            double Ex = E[c], Ey = E[n + c];
            double Bx = B[c], By = B[n + c];
            double Exl = gamma0 * (Ex + b0 * ORC_C * By);
            double Eyl = gamma0 * (Ey - b0 * ORC_C * Bx);
            double Bxl = gamma0 * (Bx - b0 * Ey / ORC_C);
            double Byl = gamma0 * (By + b0 * Ex / ORC_C);
            sum += (Exl * Byl - Eyl * Bxl) / ORC_MU0 * g->dx * g->dy;
        }
    }
    double zp = g->z0 + k_p * g->dz;
    *p_lab = sum;
    *t_lab = gamma0 * (t + b0 * zp / ORC_C);
    *z_lab = gamma0 * (zp + b0 * ORC_C * t);
}

/* ---------------------------------------------------------------------- */
/* Bunch sampling and bunching factor. */
void orc_bunch_stats(int64_t np, const double* x, const double* y, const double* z,
                     const double* ux, const double* uy, const double* uz,
                     const int32_t* lost, double k_b, double out[14]) {
    const double* v[6] = {x, y, z, ux, uy, uz};
    double s1[6] = {0, 0, 0, 0, 0, 0}, s2[6] = {0, 0, 0, 0, 0, 0};
    double re = 0.0, im = 0.0, n = 0.0;
    for (int64_t p = 0; p < np; ++p) {
        if (lost[p]) continue;
        n += 1.0;
        for (int a = 0; a < 6; ++a) {
            s1[a] += v[a][p];
            s2[a] += v[a][p] * v[a][p];
        }
        re += cos(k_b * z[p]);
        im += sin(k_b * z[p]);
    }
    for (int a = 0; a < 6; ++a) {
        double m = n > 0 ? s1[a] / n : 0.0;
        double var = n > 0 ? s2[a] / n - m * m : 0.0;
        out[a] = m;
        out[6 + a] = var > 0 ? sqrt(var) : 0.0;
    }
    out[12] = n > 0 ? sqrt(re * re + im * im) / n : 0.0;
    out[13] = n;
}

/* ---------------------------------------------------------------------- */
/* Running Fourier sums of the lab fields at a plane. */
void orc_spectrum_accumulate(const orc_grid* g, double gamma0, const double* E,
                             const double* B, int32_t k_p, double t_lab, double dt_lab,
                             int32_t n_freq, const double* omega, double* acc) {
    const int64_t n = ncell(g);
    const int64_t nv = (int64_t)(g->nx - 2) * (g->ny - 2);
    const double b0 = sqrt(1.0 - 1.0 / (gamma0 * gamma0));
    for (int m = 0; m < n_freq; ++m) {
        const double c = cos(omega[m] * t_lab) * dt_lab, s = -sin(omega[m] * t_lab) * dt_lab;
        for (int j = 1; j < g->ny - 1; ++j) {
            for (int i = 1; i < g->nx - 1; ++i) {
                int64_t q = ix(g, i, j, k_p);
                double Ex = E[q], Ey = E[n + q];
                double Bx = B[q], By = B[n + q];
                double F[4];
                F[0] = gamma0 * (Ex + b0 * ORC_C * By);
                F[1] = gamma0 * (Ey - b0 * ORC_C * Bx);
                F[2] = gamma0 * (Bx - b0 * Ey / ORC_C);
                F[3] = gamma0 * (By + b0 * Ex / ORC_C);
                double* a = acc + ((int64_t)m * nv + (int64_t)(j - 1) * (g->nx - 2) + (i - 1)) * 8;
                for (int f = 0; f < 4; ++f) {
                    a[2 * f] += F[f] * c;
                    a[2 * f + 1] += F[f] * s;
                }
            }
        }
    }
}

void orc_spectrum_density(const orc_grid* g, int32_t n_freq, const double* acc, double* out) {
    const int64_t nv = (int64_t)(g->nx - 2) * (g->ny - 2);
    for (int m = 0; m < n_freq; ++m) {
        double sum = 0.0;
        for (int64_t v = 0; v < nv; ++v) {
            const double* a = acc + ((int64_t)m * nv + v) * 8;
            /* Re(Ex By*) - Re(Ey Bx*) */
            sum += (a[0] * a[6] + a[1] * a[7]) - (a[2] * a[4] + a[3] * a[5]);
        }
        out[m] = sum * g->dx * g->dy / (ORC_MU0 * ORC_PI);
    }
}
