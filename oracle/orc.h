/*
 * orc.h -- plain FP64 CPU oracle of the MITHRA FDTD/PIC time step
 * (Fallahi, Yahaghi, Kaertner, arXiv 1612.03310).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may load this
 * library: it is linked or called only by tests/, by __graft_entry__.smoke()
 * (as the checker) and by bench.py's cpu_baseline / reference legs.  It shares
 * no code, header, constant or table with the CUDA library; even the physical
 * constants are written out again here.
 *
 * Conventions
 *   - All quantities SI, in the bunch rest frame unless a name ends in _lab.
 *   - A scalar field on the grid is an array of nx*ny*nz doubles, vertex
 *     (i,j,k) at index (k*ny + j)*nx + i (x fastest), vertex position
 *     (x0 + i*dx, y0 + j*dy, z0 + k*dz).
 *   - A 4-component potential level is 4 such arrays back to back in the order
 *     A_x, A_y, A_z, phi.  The source array holds J_x, J_y, J_z [A/m^2] and
 *     rho [C/m^3] in the same order.  E and B hold 3 arrays each (x, y, z).
 *   - Particles: absolute positions x,y,z [m] and u = gamma*beta.
 */
#ifndef MITHRA_ORACLE_H
#define MITHRA_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int32_t nx, ny, nz;
    double dx, dy, dz;
    double x0, y0, z0;      /* position of vertex (0,0,0) */
    double dt;              /* field time step */
    int32_t n_sub;          /* Boris sub-steps per field step, dt_b = dt/n_sub */
    int32_t stencil;        /* 0 = NSFD (Sec. "Numerical Dispersion"), 1 = standard */
    int32_t space_charge;   /* 0: phi is held at zero */
    int32_t boundary;       /* 1: first-order Mur everywhere; 2: second-order Mur on
                               face vertices, first order on edges and corners */
} orc_grid;

typedef struct {
    double gamma0;          /* Lorentz factor of the rest frame */
    double lambda_u;        /* lab undulator period [m] */
    double K;               /* undulator parameter */
    double z_ent_lab;       /* lab z' of the undulator entrance [m] */
    double length_lab;      /* lab length [m]; <= 0 means no exit */
    int32_t fringe;         /* 1: Neumann-shaped fringe outside [0, L] */
    int32_t type;           /* 0: static undulator; 1: optical undulator, a plane
                               wave along z (input group UNDULATOR, beam-type
                               plane-wave) */
    /* optical undulator, lab frame: vector potential A' = p A0 s(tau),
     * tau = t' - d (z' - z0)/c, a0 = e A0 / (m_e c) */
    double a0;              /* strength parameter */
    double lambda_l;        /* carrier wavelength lambda0 [m] */
    double pol_x, pol_y;    /* unit transverse polarization p */
    double z0_lab;          /* reference position of the wave [m] */
    double offset;          /* c t0 [m] */
    double variance;        /* c tau [m] */
    double cep;             /* carrier envelope phase [rad] */
    int32_t direction;      /* d = -1: the wave travels towards -z; +1: towards +z */
    int32_t signal;         /* 0 modulated Neumann, 1 modulated Gaussian,
                               2 modulated hyperbolic secant, 3 sinusoidal pulse
                               (flat-top) */
    /* seed only (input group field-initialization, type): 0 plane wave,
     * 1 Gaussian beam focused at (x0_lab, y0_lab, z0_lab) with waist radii
     * w_par along the polarization and w_perp across it (the
     * rayleigh-radius-parallel / -perpendicular parameters, read as the 1/e
     * radius of the field at the focus) */
    int32_t beam;
    double x0_lab, y0_lab;
    double w_par, w_perp;
} orc_undulator;

/* Coefficients of the update equation (Eq. updateEquation):
 * out = {A, a1, a2(=a3), a4(=a5), a6(=a7), a8}. Returns 0 when the scheme is
 * stable for the given grid and dt, 1 otherwise. */
int orc_coefficients(const orc_grid* g, double out[6]);

/* One potential update: next = level n+1 from prev (n-1), cur (n) and the
 * sources src (J^n, rho^{n+1/2}).  Interior by Eq. updateEquation, the six
 * faces by the Mur condition of order g->boundary (Sec. "First Order ABCs",
 * Sec. "Second Order ABCs"), edges and corners by the first-order one. */
void orc_potential_step(const orc_grid* g, const double* prev, const double* cur,
                        const double* src, double* next);

/* Seed field (Sec. "Seed Field"): a plane wave or Gaussian beam along z
 * given in the lab frame like the optical undulator (the same parameters,
 * orc_undulator with type 1), injected by the total-field/scattered-field technique: the
 * vertex plane k = 2 is the last of the scattered-field region (next to the
 * z = z_min boundary), k = 3 the first of the total-field region.  After the
 * update of level n+1 the stencil's coupling across the two planes is
 * corrected with the incident vector potential f^n (A components only; the
 * seed's phi is zero):
 *   k = 2:  psi' = psi - [A (a2 f_{i+1,k+1} + a2 f_{i-1,k+1} + a4 f_{j+1,k+1}
 *                           + a4 f_{j-1,k+1}) + a6 f_{k+1}]
 *   k = 3:  psi' = psi + [A (a2 f_{i+1,k-1} + ...) + a6 f_{k-1}],
 * over interior (i, j), with f^n = orc_incident_potential at the neighbour
 * vertex and t_n (a plane wave is uniform in x and y; a Gaussian beam is
 * not, so each neighbour takes its own value). */
void orc_seed_correction(const orc_grid* g, const orc_undulator* seed, double t_n,
                         double* next);

/* The incident vector potential of a seed or optical undulator at the
 * rest-frame point (x, y, z, t), out = (A_x, A_y).  Plane wave: A0 s(tau)
 * times the polarization.  Gaussian beam (beam = 1; the paper names the
 * type and its parameters but prints no formula, so this is the textbook
 * paraxial beam, one factor per transverse axis): with the lab point
 * (x, y, z', t') of the boost, zeta = d (z' - z0_lab) the distance past the
 * focus, xi and eta the offsets from (x0_lab, y0_lab) along p and along
 * z x p, and for each axis a with waist w_a: Rayleigh length
 * z_a = pi w_a^2 / lambda_l, width w_a(zeta) = w_a sqrt(1 + (zeta/z_a)^2),
 * wavefront curvature 1/R_a = zeta / (zeta^2 + z_a^2), Gouy phase
 * psi_a = atan(zeta / z_a):
 *   A = p A0 sqrt(w_xi/w_xi(zeta)) sqrt(w_eta/w_eta(zeta))
 *         exp(-xi^2/w_xi(zeta)^2 - eta^2/w_eta(zeta)^2) s~(x),
 *   x = tau - (xi^2/R_xi + eta^2/R_eta) / (2c) - offset/c,
 * s~ the signal with the carrier phase cep + (psi_xi + psi_eta)/2.  The lab
 * beam has no phi and no A_z (paraxial), so the boost leaves A_x, A_y as
 * they are. */
void orc_incident_potential(const orc_undulator* u, double x, double y, double z, double t,
                            double out[2]);

/* The same at n points (arrays of n doubles each; out holds n pairs). */
void orc_incident_potential_many(const orc_undulator* u, int64_t n, const double* x,
                                 const double* y, const double* z, const double* t,
                                 double* out);

/* E and B at t = (n+1/2) dt at the vertices [1, n-2]^3 from A^n, A^{n+1},
 * phi^n (Sec. "Field Evaluation"); all other vertices are set to zero. */
void orc_fields(const orc_grid* g, const double* lev_n, const double* lev_np1,
                double* E, double* B);

/* Undulator field in the rest frame at (y, z, t): the static undulator
 * (Eq. undulatorField) or the optical plane wave, transformed to the moving
 * frame. */
void orc_undulator_field(const orc_undulator* u, double y, double z, double t,
                         double E[3], double B[3]);

/* One Boris step (Eq. BorisScheme) for charge-to-mass ratio qm over dtb:
 * u <- u^{m+1/2} from u^{m-1/2} and the total fields. */
void orc_boris(double u[3], const double E[3], const double B[3], double qm, double dtb);

/* Advance all particles one field step (n_sub Boris steps), gathering the grid
 * E,B (Eq. fieldInterpolation) plus the undulator field, and deposit
 * J^{n+1} (at the mid point of the step) and rho^{n+3/2} into src_out, which
 * the caller zeroes.  t_half = t at the start positions.  Returns how many
 * particles were lost in this step. */
int64_t orc_push_deposit(const orc_grid* g, const orc_undulator* und, double q_macro,
                         double t_half, const double* E, const double* B,
                         int64_t np, double* x, double* y, double* z,
                         double* ux, double* uy, double* uz, int32_t* lost,
                         double* src_out);

/* rho of the particles at their present positions, added to rho_out. */
void orc_deposit_rho(const orc_grid* g, double q_macro, int64_t np, const double* x,
                     const double* y, const double* z, const int32_t* lost, double* rho_out);

/* Marks particles outside the valid region as lost; returns their number. */
int64_t orc_mark_lost(const orc_grid* g, int64_t np, const double* x, const double* y,
                      const double* z, int32_t* lost);

/* Radiated power through vertex plane k_p, lab frame, from grid E,B at time t
 * (rest frame).  Writes P [W], the lab time and the lab position of the plane. */
void orc_radiated_power(const orc_grid* g, double gamma0, const double* E, const double* B,
                        int32_t k_p, double t, double* p_lab, double* t_lab, double* z_lab);

/* Bunch sampling (Sec. "bunch-sampling" of the input groups: mean position,
 * mean momentum, position spread and momentum spread along x, y, z) and the
 * bunching factor |<exp(i k_b z)>| over the particles not lost.
 * out[0..2] mean x, y, z; out[3..5] mean ux, uy, uz; out[6..8] rms spread of
 * x, y, z; out[9..11] rms spread of ux, uy, uz; out[12] bunching factor;
 * out[13] number of particles counted.  Sums run serially in index order. */
void orc_bunch_stats(int64_t np, const double* x, const double* y, const double* z,
                     const double* ux, const double* uy, const double* uz,
                     const int32_t* lost, double k_b, double out[14]);

/* Frequency-resolved radiated power (FEL-OUTPUT radiation-power with
 * wavelengths).  The lab fields at interior vertices of plane k_p (the
 * transformation of orc_radiated_power) sampled at lab time t_lab are added
 * to running Fourier sums at the observed angular frequencies omega[m]:
 *   acc[((m * nv) + v) * 8 + 2f + {0,1}] += F_f (cos, -sin)(omega[m] t_lab) dt_lab,
 * F = (E'_x, E'_y, B'_x, B'_y), v = (j-1)(nx-2) + (i-1). */
void orc_spectrum_accumulate(const orc_grid* g, double gamma0, const double* E,
                             const double* B, int32_t k_p, double t_lab, double dt_lab,
                             int32_t n_freq, const double* omega, double* acc);

/* Energy through the plane per unit observed angular frequency from the
 * running sums (Parseval for real signals):
 *   out[m] = (1/pi) sum_v Re(E~x B~y* - E~y B~x*) dx dy / mu0   [J s]. */
void orc_spectrum_density(const orc_grid* g, int32_t n_freq, const double* acc, double* out);

/* Physical constants the oracle uses: c, e, m_e, eps0, mu0. */
void orc_constants(double out[5]);

#ifdef __cplusplus
}
#endif
#endif
