/*
 * mithra.h -- C ABI of the GB300 (sm_103a) FDTD/PIC time step of the MITHRA
 * full-wave free-electron-laser method (Fallahi, Yahaghi, Kaertner,
 * arXiv 1612.03310).
 *
 * One simulation advances, on one GPU and in the Lorentz-boosted bunch rest
 * frame:
 *   - the potentials A and phi on a 3-D vertex grid by the NSFD (or standard)
 *     central-difference update, Sec. "FDTD for Helmholtz Equation",
 *     Eq. updateEquation, with first-order Mur boundaries, Sec. "First Order
 *     ABCs";
 *   - E and B at the vertices from the potentials, Sec. "Field Evaluation";
 *   - the macroparticles by the Boris scheme (Eq. BorisScheme) in the
 *     trilinearly gathered grid field (Eq. fieldInterpolation) plus the static
 *     undulator field transformed into the rest frame (Eq. undulatorField and
 *     Sec. "Undulator Field");
 *   - the current and charge densities deposited back to the vertices,
 *     Sec. "Current Deposition", Eq. currentIntegral.
 *
 * Units are SI, rest frame, unless a name ends in _lab (laboratory frame).
 * Host arrays are double precision; a scalar field on the grid is
 * nx*ny*nz values with vertex (i,j,k) at index (k*ny + j)*nx + i (x fastest)
 * and position (x0 + i*dx, y0 + j*dy, z0 + k*dz).
 *
 * Every function returns a mithra_status.  Arrays passed in are copied and
 * never retained; output arrays are caller-allocated host memory.  Work is
 * ordered on the simulation's CUDA stream; a device-side failure is reported
 * by the first call that synchronises (mithra_sync and every call that copies
 * results to the host) and by the next mithra_step.  A failing call leaves a
 * message for mithra_last_error.  Simulations are independent: an error in
 * one does not affect another.
 */
#ifndef MITHRA_H
#define MITHRA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mithra_sim mithra_sim; /* opaque, owned by the library */

typedef enum {
    MITHRA_OK = 0,
    MITHRA_EINVAL = 1,    /* bad argument, size or layout */
    MITHRA_EUNSTABLE = 2, /* dt violates the scheme's stability condition */
    MITHRA_ENOMEM = 3,    /* device or pinned host allocation failed */
    MITHRA_ECUDA = 4,     /* a CUDA runtime call or kernel failed */
    MITHRA_ENUMERIC = 5,  /* NaN or Inf seen in a reduction */
    MITHRA_ELOST = 6,     /* a particle left the valid region (strict mode,
                             mithra_set_lost_policy) */
    MITHRA_EBUSY = 7,     /* reserved: batch slot in use */
    MITHRA_ENODEV = 8     /* no CUDA device of compute capability 10.3 */
} mithra_status;

typedef enum {
    MITHRA_P64 = 0,      /* all state and arithmetic in FP64 */
    MITHRA_P32 = 1,      /* FP32 fields and particle phase space with FP32
                            arithmetic; positions as an integer cell and an
                            FP32 fraction in it; FP64 frame clock, lab-frame
                            phase of the undulator and power accumulation;
                            the particle 1/gamma to FP32
                            rounding from an exactly summed 1 + u.u and one
                            float-float Newton step */
    MITHRA_P32_U64 = 2,  /* as MITHRA_P32, but the potential levels are kept as
                            compensated pairs (float hi + bfloat16 lo, so that
                            the rounding of a quasi-static potential no longer
                            accumulates) and the particle momenta are stored
                            in 64 bits as float-float pairs (about 2^-46
                            relative) and Boris-rotated in float-float
                            arithmetic; gamma as in MITHRA_P32 */
    MITHRA_P32_C = 3     /* as MITHRA_P32 with compensated potential levels */
} mithra_precision;

/* Field identifiers; the paper's field names (Ex .. Bz, Ax .. Az, Jx .. Jz,
 * F = phi, Q = rho) in the field-sampling group of its reference card. */
typedef enum {
    MITHRA_EX = 0, MITHRA_EY = 1, MITHRA_EZ = 2,
    MITHRA_BX = 3, MITHRA_BY = 4, MITHRA_BZ = 5,
    MITHRA_AX = 6, MITHRA_AY = 7, MITHRA_AZ = 8,
    MITHRA_JX = 9, MITHRA_JY = 10, MITHRA_JZ = 11,
    MITHRA_PHI = 12, MITHRA_RHO = 13,
    /* the previous potential level (needed to restart the leapfrog) */
    MITHRA_AX_PREV = 14, MITHRA_AY_PREV = 15, MITHRA_AZ_PREV = 16, MITHRA_PHI_PREV = 17
} mithra_field;

/* Grid and time step (Sec. "FDTD for Helmholtz Equation").
 * nx, ny, nz >= 4 vertices; boundary vertices are updated by the Mur
 * condition.  Particles live in cells [1, n-3] along each axis (the cell's
 * eight vertices and their curl/gradient neighbours must exist); a particle
 * that leaves this region is lost: flagged, counted and never pushed or
 * deposited again. */
typedef struct {
    int32_t nx, ny, nz;
    double dx, dy, dz;
    double x0, y0, z0;     /* position of vertex (0,0,0) */
    double dt;             /* field time step; particle step dt/n_sub */
    int32_t n_sub;         /* Boris sub-steps per field step, >= 1 */
    int32_t stencil;       /* 0 = NSFD (Eq. NSFDCoefficient), 1 = standard */
    int32_t boundary;      /* 1 = first-order Mur on every boundary vertex (Sec.
                              "First Order ABCs"); 2 = second-order Mur (Sec.
                              "Second Order ABCs") on face vertices, first order
                              on edge and corner vertices */
    int32_t space_charge;  /* 0: phi is held at zero */
} mithra_grid;

/* Undulator, given in the laboratory frame.  The rest frame moves with gamma0
 * along +z; a rest-frame event (z, t) is at lab position gamma0 (z + beta0 c t)
 * and lab time gamma0 (t + beta0 z / c).
 * type 0, static planar undulator (Eq. undulatorField):
 * B'_y = B0 cosh(ku y) sin(ku zeta), B'_z = B0 sinh(ku y) cos(ku zeta) with
 * zeta the lab distance past the entrance, K = e B0 lambda_u / (2 pi m c).
 * With fringe = 1 the field outside [0, length_lab] is the Neumann-shaped
 * taper of Sec. "Undulator Field" (at the exit in the distance past it).
 * length_lab <= 0: no exit.  K = 0 switches the undulator off.
 * type 1, optical undulator (input group UNDULATOR, undulator-type optical,
 * beam-type plane-wave): a plane wave along z with vector potential
 * A' = p A0 s(tau), tau = t' - direction (z' - z0_lab)/c, a0 = e A0/(m c),
 * p = (pol_x, pol_y) the unit transverse polarization (normalised by the
 * library), s the signal of the FIELD section's list with x = tau - offset/c,
 * w0 = 2 pi c / lambda_l, tau_v = variance / c, C = cos(w0 x + cep):
 *   signal 0 modulated Neumann   -4 ln2 (x/tau_v) C exp(-2 ln2 x^2/tau_v^2)
 *   signal 1 modulated Gaussian   C exp(-2 ln2 x^2/tau_v^2)
 *   signal 2 hyperbolic secant    C / cosh(x/tau_v)
 *   signal 3 sinusoidal pulse     the Gaussian for x <= 0, C for x > 0
 *                                 (flat-top)
 * E' = -dA'/dt', B' = curl A'; direction -1 travels towards -z (the
 * counter-propagating laser of the paper's examples), +1 towards +z.  The
 * beam-type gaussian-beam optical undulator is not built (beam must be 0);
 * a seed may be a Gaussian beam (mithra_set_seed). */
typedef struct {
    double gamma0;
    double lambda_u;
    double K;
    double z_ent_lab;
    double length_lab;
    int32_t fringe;
    int32_t type;         /* 0 static, 1 optical plane wave */
    double a0;            /* optical: strength parameter */
    double lambda_l;      /* optical: carrier wavelength [m] */
    double pol_x, pol_y;  /* optical: transverse polarization */
    double z0_lab;        /* optical: reference position of the wave [m] */
    double offset;        /* optical: c t0 [m] */
    double variance;      /* optical: c tau_v [m] */
    double cep;           /* optical: carrier envelope phase [rad] */
    int32_t direction;    /* optical: -1 or +1 */
    int32_t signal;       /* optical: 0..3 */
    int32_t beam;         /* seed only: 0 plane wave, 1 Gaussian beam (an
                             optical undulator must be 0) */
    double x0_lab, y0_lab;/* Gaussian beam: transverse position of the focus [m] */
    double w_par, w_perp; /* Gaussian beam: waist radii along and across p [m] */
} mithra_undulator;

/* Macroparticles, host arrays of n doubles in the rest frame at t = t0:
 * positions r^{1/2} [m] and normalised momenta u^0 = gamma*beta.  Each carries
 * charge q_macro [C] (negative for electrons) and the electron's
 * charge-to-mass ratio. */
typedef struct {
    int64_t n;
    double q_macro;
    const double *x, *y, *z;
    const double *ux, *uy, *uz;
} mithra_bunch;

/* Creates a simulation (the initial state of Sec. "Quantity Initialization":
 * Sec. "Field Initialization" with no seed, zero potentials; the bunch as
 * given, see mithra_make_bunch for Sec. "Electron Bunch Generation"):
 * validates the grid (MITHRA_EUNSTABLE if dt breaks
 * the stability condition, see mithra_check_grid), allocates device memory
 * (mithra_footprint bytes), copies the bunch, sorts it into cell tiles and
 * deposits rho^{1/2}.  Potentials start at zero at levels -1 and 0, J^0 = 0,
 * the frame clock at t0 = 0.  cuda_stream: a cudaStream_t to order all work
 * on, or NULL for a stream the library creates and owns (pass
 * cudaStreamLegacy for the legacy default stream).  On success *out
 * owns the simulation until mithra_destroy. */
mithra_status mithra_create(const mithra_grid* grid, const mithra_undulator* und,
                            const mithra_bunch* bunch, mithra_precision precision,
                            void* cuda_stream, mithra_sim** out);

/* Enqueues n >= 0 field steps on the stream and returns without waiting.
 * One step is the loop of Sec. "Finite Difference Time Domain (FDTD)" and
 * Sec. "Particle In Cell (PIC)": the potential update (Eq. updateEquation,
 * Sec. "FDTD for Scalar Potential") with the boundary (Sec. "Boundary
 * Truncation"), E and B at the vertices (Sec. "Field Evaluation"), the
 * gather (Eq. fieldInterpolation) and Boris push (Eq. BorisScheme) in the
 * grid and undulator fields (Sec. "Undulator Field"), the deposit of J and
 * rho (Sec. "Current Deposition", Eq. currentIntegral), then the re-sort of
 * the particles into cell tiles and the optional power sample.
 * With n >= 4 (and no profiling, and a stream other than the legacy or
 * per-thread default stream that the caller is not capturing itself) the
 * steps run as replays of four steps captured once as a CUDA graph per
 * parity of the level ping-pong (the remainder of n one by one); inside a
 * replay each step's re-sort but the last runs on an internal side stream
 * beside the next step's potential update.  Any later change of sampling,
 * spectrum, seed, fields or tuning re-captures them.  Returns the status of
 * work that has already finished. */
mithra_status mithra_step(mithra_sim* sim, int64_t n);

/* Waits for all enqueued work; returns its status. */
mithra_status mithra_sync(mithra_sim* sim);

/* Lost particles (a particle whose cell leaves [1, n-3] along any axis is
 * lost: flagged, counted and never pushed or deposited again; the paper does
 * not say what happens there).  strict == 0 (the default): that is all.
 * strict != 0: once a particle has been lost in a step taken after this
 * call, mithra_sync (and mithra_batch_sync for a member) returns
 * MITHRA_ELOST, and so does every later mithra_step (which then enqueues
 * nothing), with the count in mithra_last_error; the state is kept as it is
 * and the copy-out calls work as usual, so mithra_copy_particles shows which
 * particles left.  The call waits for the stream and takes the count so far
 * as its baseline; mithra_restore takes the restored count. */
mithra_status mithra_set_lost_policy(mithra_sim* sim, int32_t strict);

/* Number of field steps taken and the rest-frame time t0 + n dt. */
mithra_status mithra_time(const mithra_sim* sim, int64_t* n_steps, double* t);

/* Copies one whole field (mithra_field id) to host memory out[nx*ny*nz].
 * E and B are evaluated at t = t0 + (n - 1/2) dt from the two current
 * potential levels (zero on boundary vertices); A and phi are the newest
 * level (t0 + n dt, and phi at t0 + (n + 1/2) dt); J is J^n and rho is
 * rho^{n+1/2}, the sources of the next step. */
mithra_status mithra_copy_field(mithra_sim* sim, int32_t field, double* out);

/* Overwrites one whole field from host memory (potentials at either level or
 * a source); E and B cannot be set.  Used to restart a run or to start from a
 * prepared state. */
mithra_status mithra_set_field(mithra_sim* sim, int32_t field, const double* in);

/* Samples the fields selected by field_mask (bit f for mithra_field f < 14) at
 * npts vertices ijk[3*p .. 3*p+2] = (i, j, k).  out[p*m + s] holds the s-th
 * selected field (ascending id) at point p, m = popcount(field_mask). */
mithra_status mithra_sample_fields(mithra_sim* sim, uint32_t field_mask, const int32_t* ijk,
                                   int64_t npts, double* out);

/* Radiated power in +z through the vertex plane k_plane (1 <= k_plane <=
 * nz-2), in the laboratory frame: the grid E, B at t = t0 + (n - 1/2) dt are
 * transformed to the lab and the Poynting flux is summed over the interior
 * (i, j) in FP64.  Also returns the lab time and lab position of the plane at
 * that instant. */
mithra_status mithra_radiated_power(mithra_sim* sim, int32_t k_plane, double* p_lab,
                                    double* t_lab, double* z_lab);

/* Makes every following step also record the radiated power through k_plane
 * (FP64, on the device) for up to capacity steps; capacity 0 switches the
 * recording off.  mithra_read_power copies the records: out[3*r] = power [W],
 * out[3*r+1] = lab time, out[3*r+2] = lab position of the plane; *count
 * receives the number of records (<= max_records copied). */
mithra_status mithra_set_power_sampling(mithra_sim* sim, int32_t k_plane, int64_t capacity);
mithra_status mithra_read_power(mithra_sim* sim, double* out, int64_t max_records,
                                int64_t* count);

/* Copies the particles back in their original order (on the device the
 * library keeps them in the order of their cell tiles, each step's re-sort
 * writing the slot map the next step reads them through): positions [m],
 * momenta, and lost[p] = 1
 * for lost particles (any of the pointers may be NULL).  *n_lost receives the
 * number of lost particles. */
mithra_status mithra_copy_particles(mithra_sim* sim, double* x, double* y, double* z,
                                    double* ux, double* uy, double* uz, int32_t* lost,
                                    int64_t* n_lost);

/* Checkpoint and resume.  mithra_snapshot_bytes gives the size of a
 * snapshot; mithra_snapshot waits for the stream and copies the simulation's
 * device state (both potential levels and their lo parts, the increment, the
 * sources, the particles, the last re-sort's tile offsets, list and slot map,
 * the step counter, lost count and error word) into out (host,
 * caller-allocated, that size).  mithra_restore copies such a snapshot back into a simulation
 * created with the same grid, precision and particle count (MITHRA_EINVAL
 * otherwise, nothing changed; MITHRA_EBUSY in a batch); its undulator, seed
 * and launch choices are its own.  Recording diagnostics (power, bunch,
 * spectrum) are not part of the state and stop at a restore.  Stepping a
 * restored simulation continues the saved one (up to the order of the
 * floating-point current atomics). */
mithra_status mithra_snapshot_bytes(const mithra_sim* sim, int64_t* bytes);
mithra_status mithra_snapshot(mithra_sim* sim, void* out);
mithra_status mithra_restore(mithra_sim* sim, const void* in);

/* Frees everything the simulation owns (waits for its work first). */
mithra_status mithra_destroy(mithra_sim* sim);

/* Last error message of sim, or of the calling thread when sim is NULL.
 * The string stays valid until the next call on the same sim / thread. */
const char* mithra_last_error(const mithra_sim* sim);

/* Per-kernel timing with CUDA events recorded on the simulation's stream:
 * with enable != 0 every following step records an event pair around each
 * kernel it launches; enable == 0 stops recording.  mithra_kernel_times waits
 * for the stream and returns, per kernel id k < *n_kernels, the summed
 * duration ms[k] (milliseconds) and the number of launches[k] since
 * profiling was enabled (arrays of max_kernels entries).  mithra_kernel_name
 * names kernel id k (NULL when out of range). */
mithra_status mithra_profile(mithra_sim* sim, int32_t enable);
mithra_status mithra_kernel_times(mithra_sim* sim, double* ms, int64_t* launches,
                                  int32_t max_kernels, int32_t* n_kernels);
const char* mithra_kernel_name(int32_t kernel);

/* Source tiles the next potential update reads (Sec. "Current Deposition"
 * deposits J and rho at the vertices around each particle; the update of
 * the potentials (Eq. waveEquation) adds them).  The particle step marks
 * the 8x8x8-cell tiles (tile index ((k/8) nty + j/8) ntx + i/8 of vertex
 * (i, j, k), ntx = ceil(nx/8), nty = ceil(ny/8)) that its deposits reached,
 * and the z-marching update loads the sources of marked tiles only; the
 * sources of every other tile are zero.  *marked receives the number of
 * tiles marked for the next step, *everywhere 1 when that update reads the
 * sources of every vertex instead (after the initial deposit, a step of the
 * per-particle form, a set or restored source field, or a deposit further
 * than one tile from its particle's tile) and 0 otherwise.  Waits for the
 * simulation's stream.  Errors: MITHRA_EINVAL for a NULL argument,
 * MITHRA_ECUDA when a copy fails. */
mithra_status mithra_source_tiles(mithra_sim* sim, int64_t* marked, int32_t* everywhere);

/* Seed field (Sec. "Seed Field"; input group field-initialization),
 * injected by the total-field/scattered-field technique: wave describes a
 * wave along z in the lab frame with the parameters of an optical undulator
 * (type must be 1; its gamma0 is not used, the simulation's frame is).
 * beam 0: the plane wave A' = p A0 s(tau).  beam 1: a Gaussian beam
 * focused at (x0_lab, y0_lab, z0_lab) with waist radii w_par along p and
 * w_perp across it (the rayleigh-radius-parallel / -perpendicular
 * parameters, read as the 1/e radius of the field at the focus; the paper
 * prints no formula, this is the paraxial beam): with zeta = direction
 * (z' - z0_lab), xi and eta the lab offsets from the focus along p and
 * along z x p, and per axis z_a = pi w_a^2 / lambda_l,
 * w_a(zeta) = w_a sqrt(1 + zeta^2/z_a^2), 1/R_a = zeta / (zeta^2 + z_a^2),
 * psi_a = atan(zeta / z_a),
 *   A' = p A0 sqrt(w_xi w_eta / (w_xi(zeta) w_eta(zeta)))
 *          exp(-xi^2/w_xi(zeta)^2 - eta^2/w_eta(zeta)^2) s~(x),
 *   x = tau - (xi^2/R_xi + eta^2/R_eta)/(2c) - offset/c,
 * s~ the signal with carrier phase cep + (psi_xi + psi_eta)/2; no phi and
 * no A_z, so the boost leaves A_x and A_y as they are.  Vertex plane k = 2
 * is the last of the scattered-field region next to the z = z_min boundary,
 * k = 3 the first of the total-field region; after each update of the
 * potentials the coupling of each vertex of one plane to its neighbours on
 * the other (the z neighbour and, through the NSFD terms, its x and y
 * neighbours) is corrected with the incident vector potential of level n at
 * those neighbours, so that the seed enters the total-field region.  NULL
 * switches the seed off.  Needs nz >= 8; MITHRA_EINVAL for a bad wave;
 * MITHRA_EBUSY while the sim is in a batch. */
mithra_status mithra_set_seed(mithra_sim* sim, const mithra_undulator* wave);

/* Bunch sampling (the input group "bunch-sampling": mean position, mean
 * momentum, position spread and momentum spread along x, y, z) and the
 * bunching factor |<exp(i k_b z)>| over the particles not lost, at the
 * current state (positions r^{n+1/2}, momenta u^n).  out (host, 14 doubles):
 * out[0..2] mean x, y, z [m]; out[3..5] mean u_x, u_y, u_z; out[6..8] rms
 * spread of x, y, z; out[9..11] rms spread of u_x, u_y, u_z; out[12] the
 * bunching factor at k_b [1/m] (rest frame); out[13] the number of particles
 * counted.  FP64 sums in a fixed order; waits for the stream. */
mithra_status mithra_bunch_stats(mithra_sim* sim, double k_b, double* out);

/* Bunch sampling with time (the group's rhythm): after every `every`-th step
 * from now on, the statistics of mithra_bunch_stats at k_b are recorded on
 * the device, up to `capacity` records (every = 0 or capacity = 0 stops and
 * frees them; MITHRA_EBUSY while the sim is in a batch).  mithra_read_bunch
 * copies up to max_records records of 15 doubles each into out (host):
 * out[15 r] = the number of steps the simulation had completed at the
 * sample, out[15 r + 1 .. 15 r + 14] = the statistics; *count receives the
 * number recorded so far.  Both wait for the stream. */
mithra_status mithra_set_bunch_sampling(mithra_sim* sim, double k_b, int32_t every,
                                        int64_t capacity);
mithra_status mithra_read_bunch(mithra_sim* sim, double* out, int64_t max_records,
                                int64_t* count);

/* Frequency-resolved radiated power (FEL-OUTPUT radiation-power with
 * wavelengths).  mithra_set_spectrum starts running Fourier sums of the lab
 * fields E'_x, E'_y, B'_x, B'_y (the transformation of mithra_radiated_power)
 * at the interior vertices of vertex plane k_plane, one set per lab
 * wavelength lambda_lab[m] (host array, metres, n_wavelengths <= 64; 0 stops
 * and frees them): every following step adds the sample at lab time
 * t' = gamma0 (t + beta0 z_p / c), t = (n + 1/2) dt, weighted by
 * exp(-i w_m t') gamma0 dt, where w_m = 2 pi c (1 - beta0) / lambda_lab[m] is
 * the angular frequency at which a forward lab wave of that wavelength
 * passes the plane (which moves with the rest frame).  Device memory:
 * 64 B x (nx-2)(ny-2) per wavelength.  MITHRA_EBUSY while the sim is in a
 * batch.  mithra_read_spectrum writes, per wavelength, the energy through
 * the plane per unit of that angular frequency so far [J s],
 *   dW/dw = (1/pi) sum Re(E'~x B'~y* - E'~y B'~x*) dx dy / mu0,
 * (dW_domega: host, n_wavelengths doubles; may be NULL) and the number of
 * samples taken; it waits for the stream. */
mithra_status mithra_set_spectrum(mithra_sim* sim, int32_t k_plane, int32_t n_wavelengths,
                                  const double* lambda_lab);
mithra_status mithra_read_spectrum(mithra_sim* sim, double* dW_domega, int64_t* n_samples);

/* Launch choices (the autotuner's knobs).  Results do not depend on them
 * beyond floating-point rounding.
 *   stencil_variant 0: the direct potential update, one thread per vertex with
 *     neighbours read through L1; 1: the z-marching form, psi^n, D and source
 *     planes of a 32 x 8 column tile streamed through a shared-memory ring by
 *     TMA box loads (single-float levels only: MITHRA_P32, MITHRA_P64);
 *     2: register z-marching, a thread walks its column for lz planes with
 *     three planes' sums in registers.
 *   lz: planes per CTA of the marching forms (0: about two waves of CTAs for
 *     variant 1, 16 for variant 2).
 *   push_variant 0: one thread per particle, E and B evaluated at the eight
 *     vertices from global memory; 1: persistent CTAs over 8^3-cell particle
 *     tiles with the potentials, E/B and the deposit block in shared memory.
 *   push_ctas_per_sm: persistent CTAs per SM of push variant 1 (0: as many as
 *     fit).
 *   push_sparse_below: push variant 1 only; a tile holding fewer particles
 *     than this skips the shared-memory staging: one warp pushes its
 *     particles with E and B from global memory and deposits with global
 *     atomics, after the CTAs have taken every denser tile (0: every tile is
 *     staged).  Takes effect from the tile list of the next re-sort.
 * Defaults: stencil_variant 2 with lz 16 (the fastest form of the potential
 * update on every grid timed), push_variant 1 when the driver provides TMA
 * tensor maps (else 0), push_ctas_per_sm 0, push_sparse_below 0. */
typedef struct {
    int32_t stencil_variant;
    int32_t lz;
    int32_t push_variant;
    int32_t push_ctas_per_sm;
    int32_t push_sparse_below;
} mithra_tuning;

mithra_status mithra_set_tuning(mithra_sim* sim, const mithra_tuning* tuning);
mithra_status mithra_get_tuning(const mithra_sim* sim, mithra_tuning* tuning);

/* Radiated power through vertex plane k_plane (1 <= k_plane <= nz-2), as
 * mithra_radiated_power computes it, from caller-owned device arrays, and
 * without allocating any memory.  The paper has no counterpart: this entry
 * point exists for callers that cannot call cudaMalloc, such as an operator
 * inside another framework whose caching allocator owns the device memory
 * (a second allocator beside it fragments the device and fails once that
 * allocator has reserved the rest), or a real-time loop that must not wait
 * on the driver's allocator.
 *   psi_newest: device array of nx*ny*nz cells of 4 values {A_x, A_y, A_z,
 *     phi} of the newest potential level (float for the MITHRA_P32 forms,
 *     their hi part when compensated; double for MITHRA_P64), cell (i,j,k) at
 *     (k*ny + j)*nx + i;
 *   lo_newest: compensated forms (MITHRA_P32_C, MITHRA_P32_U64) only: device
 *     array of the level's lo parts, 4 bfloat16 per cell in the same order
 *     and layout (the level is hi + lo); NULL takes the hi parts alone, which
 *     drops the lo parts' share of E and B (a relative change of the power of
 *     order 1e-5 on the built-in workloads).  Must be NULL for MITHRA_P32 and
 *     MITHRA_P64 (MITHRA_EINVAL);
 *   increment: the same layout as psi_newest, newest minus previous level.
 *     E and B are taken at the time between the two levels.
 *   gamma0: Lorentz factor of the rest frame; *p_lab (host) receives the
 *     lab-frame power [W]; cuda_stream: stream to run on (NULL: the legacy
 *     default stream).  The call synchronises that stream and copies the
 *     result to *p_lab before it returns.
 * Scratch memory is one fixed file-scope device array of 8192 + 1 doubles
 * (64 KiB per device that loads the library, held until exit): grids with
 * ny > 8192 are rejected with MITHRA_EINVAL.  Every call looks up that
 * array's device address (cudaGetSymbolAddress, which allocates nothing) in
 * the caller's current context, so the address stays right after a
 * cudaDeviceReset or in a non-primary context; the first call in a context
 * may load the library's device code there, so make it before any stream
 * capture.  All calls on a device share the array and it keeps the last
 * call's partial sums; every call writes the entries it reads, so none needs
 * clearing, but calls whose GPU work overlaps (unordered streams) race on it:
 * order them.  Errors are reported by mithra_last_error(NULL). */
mithra_status mithra_plane_power_noalloc(const mithra_grid* grid, double gamma0,
                                         mithra_precision precision, const void* psi_newest,
                                         const void* lo_newest, const void* increment,
                                         int32_t k_plane, double* p_lab, void* cuda_stream);

/* Batched stepping (the served and batched forms): a batch advances all its
 * member simulations together, two steps per replay of one captured CUDA
 * graph (two steps return each member's ping-pong buffers to their state at
 * capture).  Two forms of the graph:
 *   - fused: a step is eight launches whatever the number of members (for
 *     every 30 members of the particle step and 96 of the grid phases one
 *     more): the boundary rest, the potential update, the power sample, the
 *     numbering of the members' tiles, the particle step, the two scan
 *     passes of the re-sort and its slot map, each one kernel over a work list
 *     that spans all members (flat block lists for the grid phases,
 *     persistent CTAs taking every member's tiles from one counter for the
 *     particle step), with each member's arguments in the launch's
 *     parameter space or a device table.  The members must share the
 *     precision form, undulator type and boundary order, use the register
 *     z-marching update and the tiled particle step, and record no seed,
 *     spectrum or bunch samples;
 *   - per member: the graph forks from the batch's stream to every member
 *     stream and runs each member's own launches, so that one member's
 *     memory-bound potential update overlaps another's particle step.
 * The graph is captured again after the membership changes, after an odd
 * step count, or after a member's launch parameters change (power sampling,
 * tuning, fields set from the host).
 * A member must have been created with its own stream (cuda_stream NULL, or
 * a non-default stream other than the batch's); while in a batch it is
 * stepped only by mithra_batch_step (mithra_step returns MITHRA_EBUSY), and
 * all other calls on it stay valid.  mithra_batch_remove orders the sim's
 * later work after the batch's; destroying a member removes it first. */
typedef struct mithra_batch mithra_batch;

mithra_status mithra_batch_create(void* cuda_stream, mithra_batch** out);
mithra_status mithra_batch_add(mithra_batch* batch, mithra_sim* sim);
mithra_status mithra_batch_remove(mithra_batch* batch, mithra_sim* sim);
/* Enqueues n steps of every member and returns without waiting. */
mithra_status mithra_batch_step(mithra_batch* batch, int64_t n);
/* Waits for the batch and returns the first failing member's status. */
mithra_status mithra_batch_sync(mithra_batch* batch);
/* mode 0: always per member; 1: fused whenever the members allow it; 2
 * (the default): fused when they allow it and their average size is below
 * 5e5 cell updates per step (a particle counted as 4), where the launches
 * dominate (measured: 256 members of 32 x 32 x 128 cells and 2000 particles
 * 3.8x faster fused; members of several million cells 2-5 % faster per
 * member).  mithra_batch_get_mode reports the form of the graph captured
 * last (1 fused, 0 per member). */
mithra_status mithra_batch_set_mode(mithra_batch* batch, int32_t fused);
/* Graph captures of the batch so far (each membership change, odd step
 * count or member parameter change costs one at the next step), how many
 * took the fused form, and their summed host time [s]; any pointer may be
 * NULL. */
mithra_status mithra_batch_stats(const mithra_batch* batch, int64_t* captures,
                                 int64_t* fused_captures, double* capture_seconds);
mithra_status mithra_batch_get_mode(const mithra_batch* batch, int32_t* fused);
int32_t mithra_batch_size(const mithra_batch* batch);
const char* mithra_batch_last_error(const mithra_batch* batch);
mithra_status mithra_batch_destroy(mithra_batch* batch);

/* Host-only checks (no GPU needed). */

/* Validates a grid: sizes, spacings, n_sub, boundary; and the stability
 * condition of the scheme.  Standard scheme: Eq. CFLcondition.  NSFD: with
 * r_l = c dt / d_l, the left side of Eq. NSFDDispersionCD times (c dt)^2 is
 * linear in sin^2(kz dz / 2), so a real omega for every wave vector needs
 * r_x^2 + r_y^2 < 1 and r_z <= 1.  This is the bound of the interior
 * scheme; the Mur boundaries are not stable over all of it: random
 * potentials grow within a few hundred steps for first-order faces at
 * r_z >= 0.97 with r_x^2 + r_y^2 >= 0.7 (>= 0.5 at r_z = 1), and for either
 * order at r_z = 0.8 with r_x^2 + r_y^2 >= 0.8; at r_z = 0.95 both orders
 * stayed bounded up to r_x^2 + r_y^2 = 0.97. */
mithra_status mithra_check_grid(const mithra_grid* grid);

/* Device bytes mithra_create will allocate for this grid, particle count and
 * precision (used for admission by memory footprint). */
mithra_status mithra_footprint(const mithra_grid* grid, int64_t n_particles,
                               mithra_precision precision, int64_t* bytes);

/* Library version: major*10000 + minor*100 + patch. */
int32_t mithra_version(void);

/* Lab-frame description of an FEL case and the rest-frame numbers the
 * library takes (Sec. "Lorentz Boost"; host only, FP64, no GPU needed). */
typedef struct {
    double gamma;             /* beam Lorentz factor in the lab */
    double sigma_gamma_rel;   /* rms energy spread over gamma */
    double lambda_u;          /* undulator period [m] */
    double K;                 /* undulator parameter */
    int32_t steps_per_period; /* time steps per rest-frame undulator period */
    double courant;           /* c dt / dz, in (0, 1] */
} mithra_lab_case;

typedef struct {
    double gamma0, beta0;     /* the frame: gamma / sqrt(1 + K^2/2) */
    double dt, dz;            /* rest-frame time step [s] and longitudinal cell [m] */
    double uz_mean, uz_sigma; /* the beam's mean longitudinal u = gamma beta in the
                                 frame, and the spread the lab energy spread maps to */
    double k_b;               /* rest-frame ponderomotive (bunching) wavenumber [1/m] */
    double lambda_r_lab;      /* resonant wavelength lambda_u (1 + K^2/2) / (2 gamma^2) */
} mithra_rest_frame;

/* Fills *out from *lab: gamma0 = gamma / sqrt(1 + K^2/2), c dt = (lambda_u /
 * gamma0) / steps_per_period, dz = c dt / courant; the beam's rest-frame
 * Lorentz factor gamma gamma0 (1 - beta beta0) gives uz_mean, and the lab
 * spread sigma_gamma_rel gamma scales by gamma0 (1 - beta beta0) to uz_sigma;
 * k_b = gamma0 (2 pi / lambda_u)(1 + beta0).  MITHRA_EINVAL for gamma <= 1,
 * lambda_u <= 0, K < 0, steps_per_period < 1, courant outside (0, 1], or a
 * beam slower than the frame (gamma0 < 1 is impossible by construction). */
mithra_status mithra_boost_from_lab(const mithra_lab_case* lab, mithra_rest_frame* out);

/* Synthetic bunch in the rest frame (Sec. "Electron Bunch Generation";
 * input group bunch-initialization, type ellipsoid; host only, FP64, no GPU
 * needed).  Uniform numbers come from the Halton sequence (sequence 1, the
 * paper's loader: point i + 1 of the radical inverses in the primes 2 .. 23,
 * one prime per coordinate) or from a counter-based SplitMix64 generator
 * keyed by seed (sequence 0).  Per particle:
 *   - (x, y) = (x0, y0) + (sigma_x, sigma_y) sqrt(-2 ln a) (cos, sin)(2 pi b)
 *     (Eq. gaussian2D), drawn again while the distance from (x0, y0) exceeds
 *     trunc_r (trunc_r <= 0: no truncation; transverse-truncation);
 *   - z uniform in [z_lo, z_hi] (Eq. uniform1D); with taper_sigma > 0 a share
 *     sqrt(2 pi) taper_sigma / (z_hi - z_lo + sqrt(2 pi) taper_sigma) of the
 *     particles instead forms a Gaussian of rms taper_sigma of the same peak
 *     density, its lower half placed behind z_lo and its upper half ahead of
 *     z_hi (the smooth head and tail that avoid coherent emission at the
 *     edges of a uniform profile);
 *   - with bf > 0, z -> z - (2 bf / kb) sin(kb z), which gives
 *     |<exp(i kb z)>| = J_1(2 bf) = bf (1 - bf^2/2 + ...) for a uniform
 *     profile over whole periods (Eq. bunchingFactor; its
 *     printed form is not dimensionally consistent, and kb is the caller's
 *     rest-frame ponderomotive wavenumber, gamma0 ku (1 + beta0) for the
 *     static undulator, mithra_rest_frame.k_b);
 *   - (u_x, u_y) Gaussian of rms (ux_sigma, uy_sigma) (Eq. gaussian2D) and
 *     u_z Gaussian of mean uz_mean and rms uz_sigma (Eq. gaussian1D).
 * x .. uz: host arrays of n doubles, written; *q_macro (may be NULL)
 * receives -charge / n, the electron macroparticle charge for
 * mithra_bunch.  MITHRA_EINVAL for n < 1, z_hi < z_lo, a negative spread,
 * bf outside [0, 1) or bf > 0 without kb > 0, or a truncation that rejects
 * nearly every draw (message in mithra_last_error(NULL)). */
typedef struct {
    int64_t n;
    double charge;               /* total charge [C], > 0 (electrons) */
    double x0, y0;               /* transverse centre [m] */
    double sigma_x, sigma_y;     /* rms transverse size [m] */
    double trunc_r;              /* transverse truncation radius [m], <= 0: none */
    double z_lo, z_hi;           /* uniform longitudinal extent [m] */
    double taper_sigma;          /* rms of the head/tail Gaussian [m], 0: none */
    double ux_sigma, uy_sigma;   /* rms transverse momenta (u = gamma beta) */
    double uz_mean, uz_sigma;    /* longitudinal momentum mean and rms */
    double bf, kb;               /* bunching factor and its wavenumber [1/m] */
    int32_t sequence;            /* 0 SplitMix64 (counter-based), 1 Halton */
    uint64_t seed;               /* sequence 0 only */
} mithra_bunch_spec;

mithra_status mithra_make_bunch(const mithra_bunch_spec* spec, double* x, double* y, double* z,
                                double* ux, double* uy, double* uz, double* q_macro);

#ifdef __cplusplus
}
#endif
#endif /* MITHRA_H */
