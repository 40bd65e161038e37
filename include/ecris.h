/*
 * ecris.h - C ABI of the GB300 (sm_103a) ECRIS ion time step.
 *
 * The library advances the macroparticles of the particle-in-cell /
 * Monte-Carlo-collision model of Mironov et al., "Numerical model of Electron
 * Cyclotron Resonance Ion Source" (arXiv:1507.03392, Sec. II).  One time step
 * of one run is, in the paper's order:
 *   push        Boris push of ions in the static minimum-B field (solenoid
 *               mirror plus the printed analytic hexapole) and the electric
 *               field interpolated from a cell-centred 3-D grid; atoms move in
 *               straight lines (Sec. II, particle-in-cell tracing);
 *   MCC         step-wise electron-impact ionisation Q -> Q+1 from the cell's
 *               electron density and temperature, charge exchange with the
 *               neutral background, the electron-ion heating kick (equation for
 *               D with the delta stencil), and Takizawa-Abe / Nanbu ion-ion
 *               Coulomb collisions (Sec. II, collision block);
 *   boundaries  neutralisation and cosine-law re-emission at the walls;
 *               extraction through the round aperture at z = L with
 *               reinjection at the gas inlet, so N stays constant (Sec. II);
 *   deposition  nearest-grid-point count and charge per cell (Sec. II: the
 *               electron density equals the ion charge density).
 *
 * Conventions for every entry point:
 *   - Units are SI (m, s, m/s, T, V/m) except where a name says cm^-3, cm^2
 *     or eV.  The injection flange is at z = 0, the extraction flange at z = L;
 *     the mesh spans [-R0, R0] x [-R0, R0] x [0, L] with cell index
 *     c = (iz * ny + iy) * nx + ix (x fastest).
 *   - Every call returns an ecris_status; nothing is thrown or aborted across
 *     the ABI.  ecris_last_error() describes the last failure on a context.
 *   - Inputs are validated before any device work; an invalid argument leaves
 *     the context unchanged and returns ECRIS_EINVAL.
 *   - The library owns all device memory it allocates (stream-ordered, on the
 *     context's stream).  Pointers passed in are only read during the call
 *     (host memory) or until the call's stream work completes (device memory);
 *     the caller keeps ownership.
 *   - Calls on one context must not run concurrently from several host
 *     threads.  Device work is ordered on the context's stream; calls that
 *     return data to the host synchronise that stream.
 */
#ifndef ECRIS_H
#define ECRIS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ecris_ctx ecris_ctx;

typedef enum {
    ECRIS_OK = 0,
    ECRIS_EINVAL = 1,   /* invalid argument; nothing was changed */
    ECRIS_ENOMEM = 2,   /* device or host allocation failed */
    ECRIS_ECUDA = 3,    /* a CUDA call failed; the message names it */
    ECRIS_ETIMEOUT = 4, /* a bounded device wait ran out */
    ECRIS_ESTATE = 5    /* call out of order (e.g. step before load), or the
                           context is unusable after an earlier device error */
} ecris_status;

/* Process switches (ecris_mcc.flags). */
#define ECRIS_F_PUSH (1u << 0)    /* move particles (off: positions frozen, 0-D tests) */
#define ECRIS_F_IONIZE (1u << 1)  /* electron-impact ionisation Q -> Q+1 */
#define ECRIS_F_CX (1u << 2)      /* charge exchange with the neutral background */
#define ECRIS_F_EIKICK (1u << 3)  /* electron-ion heating / diffusion kick */
#define ECRIS_F_COULOMB (1u << 4) /* ion-ion Coulomb collisions */
#define ECRIS_F_RECYCLE (1u << 5) /* re-emit at walls, reinject extracted particles;
                                     off: leavers are frozen and counted once */
/* Opt-in processes and variants (Sec. II collision block; Secs. III.C, IV). */
#define ECRIS_F_ISOHEAT (1u << 6) /* isotropic heating: the kick without the drift
                                     bias, delta = 0 (the paper's diffusion-off run) */
#define ECRIS_F_DOUBLE (1u << 7)  /* multiple ionisation: Q -> Q+2 at k2_factor times
                                     the Lotz-Maxwellian rate with threshold
                                     P_Q + P_{Q+1}, and, when k3_factor > 0, Q -> Q+3
                                     at k3_factor times that of P_Q + P_{Q+1} + P_{Q+2};
                                     one word decides, single below p k1/k, double
                                     below p (k1+k2)/k, triple up to p = 1 - exp(-n_e
                                     k dt), k = k1 + k2 + k3 */
#define ECRIS_F_ELASTIC (1u << 8) /* elastic ion-atom scattering on the background,
                                     cross section sigma_el1_cm2 * Q, isotropic in
                                     the centre-of-mass frame with an atom drawn at
                                     T0; shares its word with charge exchange in
                                     proportion to the cross sections */
#define ECRIS_F_RECOMB (1u << 9)  /* radiative recombination Q -> Q-1 at Seaton's
                                     hydrogenic rate for charge Q and T_e; shares
                                     the ionisation word in proportion to the rates */

/* Per-particle state word (ecris_get_state meta): bits 0-7 charge state Q,
 * bits 8-15 events of the last step, bits 16-23 status. */
#define ECRIS_META_Q(m) ((m) & 0xFFu)
#define ECRIS_EV_WALL (1u << 8)     /* hit the wall (neutralised, re-emitted) */
#define ECRIS_EV_EXTRACT (1u << 9)  /* left through the aperture (reinjected) */
#define ECRIS_EV_IONIZE (1u << 10)  /* ionised this step */
#define ECRIS_EV_CX (1u << 11)      /* charge exchange this step */
#define ECRIS_EV_COULOMB (1u << 12) /* took part in a Coulomb collision */
#define ECRIS_EV_ELASTIC (1u << 13) /* elastic ion-atom scattering this step */
#define ECRIS_EV_RECOMB (1u << 14)  /* recombined this step */
#define ECRIS_ST_FROZEN (1u << 16)  /* left the chamber with recycling off */

/* Chamber geometry (Sec. II, Table I shapes). */
typedef struct {
    double R0;       /* chamber radius, m (> r_ap) */
    double L;        /* chamber length, m */
    double r_ap;     /* extraction aperture radius, m (> 0) */
    double inlet[3]; /* gas inlet point where extracted particles are reinjected, m;
                        must lie inside the chamber */
} ecris_geometry;

/* Static magnetic field (Sec. II, Fig. 3 extremes and the hexapole equations).
 * The solenoid maps of the paper are not available: the on-axis profile is a
 * synthetic mirror through B_inj (z=0), B_min (at z_m) and B_ext (z=L) made of
 * raised-cosine halves with continuous second derivative, extended off axis
 * by the paraxial expansion B_r = -(r/2) B0', B_z = B0 - (r^2/4) B0''.  The
 * hexapole adds B_x = B_H sin(2 theta) R^2/R0^2, B_y = B_H cos(2 theta) R^2/R0^2. */
typedef struct {
    double B_inj, B_min, B_ext; /* T; B_inj > B_min >= 0, B_ext > B_min */
    double B_hex;               /* hexapole field at r = R0, T */
    double B_ecr;               /* resonance field, T (0.5 T at 14 GHz) */
    /* Optional on-axis table replacing the synthetic mirror (a computed
     * solenoid map, the flat or middle-coil profiles of Sec. IV): B0 at
     * n_axial points z_k = k L / (n_axial - 1), host memory, copied.  The
     * library takes the natural cubic spline through the samples for B0, B0'
     * and B0'' and extends it off axis as above.  n_axial = 0: the mirror
     * (B_inj, B_min, B_ext are then required); otherwise 4 <= n_axial <= 65537
     * finite samples >= 0. */
    int32_t n_axial;
    const double* B_axial;
} ecris_bfield;

/* Mesh and electron background (Sec. II: 3-D Cartesian mesh; warm electrons
 * T_ew inside the ECR zone, cold T_ec outside; n_e per cell).  A cell is in
 * the zone when |B| at its centre is below B_ecr. */
typedef struct {
    int32_t nx, ny, nz;        /* cells, each >= 2 */
    const float* E;            /* host, 3*Nc floats (Ex,Ey,Ez per cell centre, V/m),
                                  or NULL for E = 0 (the paper's case) */
    double ne_in_cm3;          /* n_e inside the zone, cm^-3 (when ne_in_cells == NULL) */
    const float* ne_in_cells;  /* host, Nc floats, cm^-3: per-cell n_e used inside the
                                  zone; may be NULL */
    double ne_out_cm3;         /* n_e outside the zone, cm^-3 */
    double Te_warm_eV;         /* T_ew, eV (> 0) */
    double Te_cold_eV;         /* T_ec, eV (> 0) */
} ecris_grid;

/* Ion species.  The paper's rate datasets [20-23] are not available: the
 * library builds the rate of Q -> Q+1 as the Maxwellian average of the
 * single-term Lotz cross section from the ionisation potential P_Q and the
 * number of outer electrons q_Q. */
typedef struct {
    double mass_amu;           /* > 0 */
    int32_t qmax;              /* highest charge state, 1..63 */
    const double* ip_eV;       /* host, qmax values: P_Q for Q = 0..qmax-1 (> 0) */
    const int32_t* n_outer;    /* host, qmax values: q_Q >= 1 */
} ecris_species;

/* Collisions and switches (Sec. II collision block). */
typedef struct {
    double n0_cm3;          /* neutral background density for charge exchange, cm^-3 */
    double T0_eV;           /* gas / wall temperature, eV (0.025-0.026) */
    double sigma1_cm2;      /* charge-exchange cross section of Q=1 (scaled by Q), cm^2 */
    double E_cx_eV;         /* charge-exchange energy release (10 eV), half to the ion */
    double lnL_ii;          /* ion-ion Coulomb logarithm (10) */
    double lnL_ei;          /* electron-ion Coulomb logarithm (17) */
    int32_t ei_charge_power;/* 1 or 2: power of Q in the kick's D^2 (2 = the text's
                               quadratic dependence) */
    uint32_t flags;         /* ECRIS_F_* */
    double T_refl_eV;       /* re-emission temperature of ions neutralised at a wall
                               (Sec. III.C warm atoms, 0.15 eV); 0: T0 */
    double sigma_el1_cm2;   /* elastic ion-atom cross section of Q=1, cm^2 (ECRIS_F_ELASTIC) */
    double k2_factor;       /* double-ionisation rate factor (ECRIS_F_DOUBLE), >= 0 */
    double k3_factor;       /* triple-ionisation rate factor (ECRIS_F_DOUBLE), >= 0; 0: none */
} ecris_mcc;

/* Diagnostics filled by ecris_diag.  Arrays are caller-owned; each array
 * pointer may be NULL to skip it; lengths are stated per field. */
typedef struct {
    int32_t qmax;             /* out: the run's qmax */
    uint64_t steps;           /* out: steps since ecris_load_ions */
    double time_s;            /* out: simulated time since load (sum of dt) */
    int64_t* extracted;       /* qmax+1: particles that left through the aperture, per Q */
    int64_t* lost;            /* qmax+1: wall hits, per Q at the hit */
    int64_t* alive_by_q;      /* qmax+1: current census of particles in the chamber */
    double* current_A;        /* qmax+1: extracted current Q e w count / time (Sec. III) */
    double ke_lost_eV;        /* out: kinetic energy of ions (Q >= 1) that left, per
                                 macroparticle, summed (multiply by the weight for real ions) */
    double power_W;           /* out: power balance of Sec. II over the time since load:
                                 w * sum over ions that left of (kinetic + ionisation
                                 potential energy + Q * 3/2 T_ew) / time */
    int64_t coulomb_collisions; /* out: pair collisions performed */
    uint64_t* cell_count;     /* Nc: time-summed NGP particle counts per cell */
    uint64_t* cell_charge;    /* Nc: time-summed NGP charge (sum of Q) per cell */
} ecris_diag_out;

/* Create a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t
 * to order all work on, or NULL to let the library create its own.  On
 * success *out receives the context. */
ecris_status ecris_create(ecris_ctx** out, int device, void* cuda_stream);

/* Release the context and all device memory it owns (synchronises its stream). */
void ecris_destroy(ecris_ctx* ctx);

/* Message for the last failure on ctx (empty string if none); valid until the
 * next call on ctx.  ctx may be NULL (then describes the last failure of
 * ecris_create or ecris_coulomb_collide_noalloc on this thread). */
const char* ecris_last_error(const ecris_ctx* ctx);

/* Per-run setup (Sec. II model inputs): validates the inputs, builds in FP64
 * on the host the ionisation rates for T_ew and T_ec, the ECR zone, n_e and the
 * delta vector of every cell (printed 3x3 stencil scaled by
 * R_L = 2.38e-6 sqrt(T_e)/(B dX)), and copies them and the E grid to the device.
 * Must precede ecris_load_ions; calling it again replaces the fields and
 * requires a new ecris_load_ions. */
ecris_status ecris_init_fields(ecris_ctx* ctx, const ecris_geometry* geo, const ecris_bfield* bf,
                               const ecris_grid* grid, const ecris_species* sp,
                               const ecris_mcc* mcc);

/* Load n macroparticles (Sec. II: position, velocity, charge state, weight).
 * xyzv[0..5] point to n floats each: x, y, z (m), vx, vy, vz (m/s); q to n
 * bytes (Q, 0 = atom, <= qmax).  Host pointers when src_is_device == 0,
 * device pointers otherwise.  Positions must lie inside the chamber.
 * weight: real particles per macroparticle (> 0).  seed: key of the
 * counter-based random numbers (Philox4x32-10 with counter (particle, 0,
 * 4*step + stream, 0)).  Copies the data; resets tallies, deposit grids and the
 * step counter.  n may be 0.  n * max(qmax, 1) must stay below 2^32. */
ecris_status ecris_load_ions(ecris_ctx* ctx, size_t n, const float* const xyzv[6], const uint8_t* q,
                             double weight, uint64_t seed, int src_is_device);

/* Advance nsteps time steps of length dt (s, > 0).  Asynchronous on the
 * context's stream.  The total step count since load must stay below 2^30. */
ecris_status ecris_step(ecris_ctx* ctx, uint32_t nsteps, double dt);

/* Copy the diagnostics of the run to caller memory (synchronises). */
ecris_status ecris_diag(ecris_ctx* ctx, ecris_diag_out* out);

/* Self-consistent electron density (Sec. II: the electron density equals the
 * ion charge density, by charge neutrality).  Replaces the prescribed n_e of
 * every cell by the time-averaged ion charge density since the load or the
 * previous call:
 *     n_e(c) = w * sum over steps and particles in c of Q / (steps * V_cell),
 * with w the load's weight, V_cell = (2 R0/nx)(2 R0/ny)(L/nz) and the
 * deposit that ecris_diag reports as cell_charge (ions after each step's
 * move, NGP), and rebuilds each cell's delta from it (the 3x3 stencil and
 * R_L of the heating kick, Sec. II).  The zones (warm / cold electrons) stay
 * as |B| gave them.  Cells without ions get n_e = 0 (no ionisation, no
 * heating).  Runs on the device in stream order after the queued steps and
 * returns without waiting (nothing is read back).  ECRIS_ESTATE when no step
 * ran since the load or the previous call; the run is unchanged then. */
ecris_status ecris_update_ne(ecris_ctx* ctx);

/* First-passage time distribution (Sec. III.D): for every ion extracted
 * through the aperture, its age in steps since the particle was last
 * ionised from Q = 0 (an ion loaded as an ion, whose birth is unknown, is not
 * counted; a particle neutralised at a wall or by charge exchange starts a
 * new age at its next ionisation).  Ages a >= 1 are binned by
 *     e = floor(log2 a),  m = the two bits of a below its leading one
 *     (a << (2 - e) & 3 for e < 2),  bin = 4 e + m,
 * so bin 4e + m starts at a = 2^e (1 + m/4) for e >= 2.  Multiply by dt for
 * seconds. */
#define ECRIS_FPTD_BINS 120

/* Copy the distribution out: hist[(qmax + 1) * ECRIS_FPTD_BINS] counts by
 * (Q, bin), row Q = 0 empty; age_sum[qmax + 1] the summed ages (steps) by Q,
 * for the mean.  Either pointer may be NULL.  Host memory; synchronises.
 * Counts since the load. */
ecris_status ecris_get_fptd(ecris_ctx* ctx, uint64_t* hist, uint64_t* age_sum);

/* Summed radius sqrt(x^2 + y^2) of the extracted ions at the aperture
 * plane, by charge state, in metres (accumulated in whole nanometres since
 * the load); the mean radial displacement of Sec. III.A is
 * r_sum[Q] / extracted[Q].  r_sum holds qmax + 1 values.  Synchronises. */
ecris_status ecris_get_extraction_radius(ecris_ctx* ctx, double* r_sum);

/* Moment probes and screens (diagnostics of Sec. III.A, Figs. 9-16).  Each
 * ecris_probe_sample call adds the particles as they are now:
 *  - for every probed cell c and charge state Q (atoms Q = 0 included): the
 *    number of particles and the sums of vx, vy, vz, vx^2, vy^2, vz^2, in
 *    FP64; the density of Q in c is w count / (samples V_cell) and its
 *    temperature M (<v^2> - <v>^2) / 3 in energy units (the ion pressure of
 *    a cell is the sum over Q of n_Q T_Q, its mean temperature that pressure
 *    over the summed density);
 *  - for every screen s, a slab z_lo[s] <= z < z_hi[s]: a hit on the pixel
 *    under each particle in the slab, by Q, on a pixels x pixels grid over
 *    the square [-R0, R0)^2 (pixel (px, py) covers x from -R0 + 2 R0 px /
 *    pixels, row-major with px fastest).
 * Sampled every step, the screens are the paper's exposure images (a pixel
 * counts a particle each time step it is there); sampled every k steps they
 * estimate the same picture at 1/k of the counts. */
#define ECRIS_MAX_SCREENS 4
typedef struct {
    size_t ncells;            /* probed cells, each at most once */
    const uint32_t* cells;    /* their indices (ix fastest), host memory */
    int32_t nscreens;         /* 0 .. ECRIS_MAX_SCREENS */
    double z_lo[ECRIS_MAX_SCREENS], z_hi[ECRIS_MAX_SCREENS];   /* slabs (m), 0 <= z_lo < z_hi <= L */
    int32_t pixels;           /* power of two, 2 .. 4096 (ignored without screens) */
} ecris_probe_spec;

/* Install the probes (replacing earlier ones) and zero their sums; a load
 * zeroes them as well.  Needs ecris_init_fields.  ECRIS_EINVAL for a cell
 * index out of range, a repeated cell, a bad slab or pixel count. */
ecris_status ecris_set_probes(ecris_ctx* ctx, const ecris_probe_spec* spec);
/* Add the current particles (asynchronous on the context's stream). */
ecris_status ecris_probe_sample(ecris_ctx* ctx);
/* Copy the sums out (synchronises); any pointer may be NULL:
 *   samples     number of ecris_probe_sample calls since the sums were zeroed;
 *   moments     [ncells][qmax + 1][7]: count, sum vx, vy, vz, sum vx^2, vy^2, vz^2;
 *   screens     [nscreens][qmax + 1][pixels * pixels] hit counts. */
ecris_status ecris_get_probes(ecris_ctx* ctx, uint64_t* samples, double* moments, uint64_t* screens);

/* Copy the per-cell electron data the kernels read to host memory: n_e in
 * m^-3 and the two delta components, nx*ny*nz floats each in cell order
 * (ix fastest); any pointer may be NULL.  Synchronises. */
ecris_status ecris_get_cells(ecris_ctx* ctx, float* ne, float* delta_x, float* delta_y);

/* Copy the particle state out: xyzv[0..5] n floats each, meta n words (see
 * ECRIS_META_Q / ECRIS_EV_* / ECRIS_ST_*), any pointer may be NULL.  Host
 * pointers when dst_is_device == 0 (synchronises), device pointers otherwise
 * (ordered on the context's stream). */
ecris_status ecris_get_state(ecris_ctx* ctx, float* const xyzv[6], uint32_t* meta, int dst_is_device);

/* Kernel timing (tracing aid, not part of the paper's model).  When enabled,
 * every kernel launch of ecris_step on the context's stream is bracketed by
 * CUDA events; ecris_get_profile synchronises and reports, per kernel kind,
 * the number of launches and their summed device time since the last reset. */
typedef struct {
    int64_t step_launches;     /* fused push/MCC/boundary/deposit kernel */
    double step_ms;
    int64_t coulomb_launches;  /* ion-ion collision kernels (binning, pairing; one run's leaver
                                  pass runs inside them when the run has collisions) */
    double coulomb_ms;
    int64_t other_launches;    /* leaver pass of runs without collisions, sorts, deposit fold and
                                  bookkeeping kernels */
    double other_ms;
} ecris_profile;

/* enable != 0 turns timing on (and resets the counters), 0 turns it off */
ecris_status ecris_set_profiling(ecris_ctx* ctx, int enable);
ecris_status ecris_get_profile(ecris_ctx* ctx, ecris_profile* out);

/* Performance knobs (not part of the paper's model; results do not depend on
 * them).  The library keeps each run's particles grouped by (ion or atom,
 * cell) in device memory and regroups them every sort_every steps (default
 * 32; >= 1).  ecris_get_state always returns particles in load order. */
typedef struct {
    int32_t sort_every;
    int32_t blocks_per_sm;  /* batches: resident step-kernel blocks per SM (0: as many as fit) */
    int32_t threads;        /* batches: step-kernel threads per block, 128, 256 or 512 (0: 256) */
    int32_t particles_per_thread;   /* batches: particles per thread and tile, 1, 2 or 4 (0: 2) */
    int32_t stages;         /* batches: tiles held in shared memory per block, 2 or 3 (0: 3 where the
                               shape has a three-stage form, else 2) */
    int32_t reserved[3];    /* set to 0 */
} ecris_tuning;
ecris_status ecris_set_tuning(ecris_ctx* ctx, const ecris_tuning* t);

/* ------------------------------------------------------------------------ */
/* Batched form: many runs advanced together (the paper's parameter scans of */
/* Sec. III -- gas flow, microwave power via n_e and T_e -- run as one       */
/* batch).  Every step of all active runs is one persistent launch of the     */
/* step kernel over a work list of (run, tile) items, captured with the       */
/* runs' collision kernels in one CUDA graph.  Each run keeps its particles   */
/* resident on the device and gives exactly the results it gives alone.      */
/* ------------------------------------------------------------------------ */
typedef struct ecris_batch ecris_batch;

/* Create a batch on `device`, ordering its work on `cuda_stream` (NULL: its
 * own stream).  hbm_budget_bytes > 0 caps the device memory the batch's runs
 * may hold (see ecris_run_bytes); 0 means no cap. */
ecris_status ecris_batch_create(ecris_batch** out, int device, void* cuda_stream, size_t hbm_budget_bytes);
void ecris_batch_destroy(ecris_batch* b);
/* message for the last failure on the batch (empty if none) */
const char* ecris_batch_last_error(const ecris_batch* b);

/* Device bytes a run of n particles on an nx x ny x nz mesh holds in a batch
 * (an upper estimate used for admission). */
size_t ecris_run_bytes(size_t n, int32_t nx, int32_t ny, int32_t nz, int coulomb);

/* Add a run: the arguments of ecris_init_fields and ecris_load_ions plus its
 * time step dt (s).  On success *run_out receives the run's handle (>= 0).
 * Returns ECRIS_ENOMEM without side effects when the run would exceed the
 * batch's memory budget (the caller may retry after removing runs). */
ecris_status ecris_batch_add_run(ecris_batch* b, const ecris_geometry* geo, const ecris_bfield* bf,
                                 const ecris_grid* grid, const ecris_species* sp, const ecris_mcc* mcc,
                                 size_t n, const float* const xyzv[6], const uint8_t* q, double weight,
                                 uint64_t seed, double dt, int src_is_device, int32_t* run_out);
/* Remove a run and release its device memory (synchronises the stream). */
ecris_status ecris_batch_remove_run(ecris_batch* b, int32_t run);
/* Advance every run of the batch by nsteps steps of its own dt. */
ecris_status ecris_batch_step(ecris_batch* b, uint32_t nsteps);
/* Per-run diagnostics and state, as ecris_diag / ecris_get_state. */
ecris_status ecris_batch_diag(ecris_batch* b, int32_t run, ecris_diag_out* out);
ecris_status ecris_batch_get_state(ecris_batch* b, int32_t run, float* const xyzv[6], uint32_t* meta,
                                   int dst_is_device);
/* ecris_update_ne / ecris_get_cells for one run of the batch, ordered after
 * its queued steps on the batch stream (the update does not wait; reading
 * the cells does). */
ecris_status ecris_batch_update_ne(ecris_batch* b, int32_t run);
ecris_status ecris_batch_get_fptd(ecris_batch* b, int32_t run, uint64_t* hist, uint64_t* age_sum);
ecris_status ecris_batch_get_extraction_radius(ecris_batch* b, int32_t run, double* r_sum);
ecris_status ecris_batch_set_probes(ecris_batch* b, int32_t run, const ecris_probe_spec* spec);
ecris_status ecris_batch_probe_sample(ecris_batch* b, int32_t run);
ecris_status ecris_batch_get_probes(ecris_batch* b, int32_t run, uint64_t* samples, double* moments,
                                    uint64_t* screens);
ecris_status ecris_batch_get_cells(ecris_batch* b, int32_t run, float* ne, float* delta_x, float* delta_y);
/* Bytes held by the batch's runs and its budget (0: none). */
ecris_status ecris_batch_memory(const ecris_batch* b, size_t* used, size_t* budget);
/* Kernel timing for a batch, as ecris_set_profiling / ecris_get_profile:
 * with profiling on, every step launches its kernels one by one (no graph)
 * between events; step_* is the batched step kernel, coulomb_* the collision
 * kernels of all runs, other_* sorts, deposit folds and step counters. */
ecris_status ecris_batch_set_profiling(ecris_batch* b, int enable);
ecris_status ecris_batch_get_profile(ecris_batch* b, ecris_profile* out);
/* Launch-shape autotuner.  Times `trial_steps` steps of the batch (no sort
 * among them) in each launch shape of the step kernel -- threads per block
 * 128, 256 or 512 times particles per thread 1, 2 or 4 with two stages, and
 * 128 x 2, 256 x 1 and 256 x 2 with three -- with as many resident blocks as
 * fit; then, in the fastest shape, each count of resident
 * blocks per SM; then each sort cadence (8, 32, 128, 256, 512 steps), in whole sort
 * periods that each start with a sort.  Keeps the fastest of each and returns
 * the choice in *chosen (may be NULL).  Before the trials every run's state
 * (particles, tallies, deposit and time sums, first-passage records, step
 * counter) is copied aside in device memory, and it is restored afterwards:
 * the trials use no simulated time, and the runs continue from where they
 * were.  ECRIS_ENOMEM if that copy does not fit (nothing is changed then).
 * No result depends on the choice. */
ecris_status ecris_batch_autotune(ecris_batch* b, uint32_t trial_steps, ecris_tuning* chosen);
/* Set the batch's tuning directly (the fields of ecris_tuning: sort_every >= 1,
 * blocks_per_sm >= 0, threads x particles_per_thread x stages one of the
 * shapes above, or threads and particles_per_thread both 0 for 256 x 2 with
 * three stages; ECRIS_EINVAL otherwise).  No result depends on it. */
ecris_status ecris_batch_set_tuning(ecris_batch* b, const ecris_tuning* t);

/* ------------------------------------------------------------------------ */
/* Served form: a request loop (a library thread) that keeps a batch on the  */
/* device and admits submitted runs as slots and memory free up (continuous  */
/* batching).  A run is stepped until its extracted currents converge (Sec.  */
/* II: the model's results hold for the stationary state of the source) or  */
/* a step cap, then retired.  The rule is checked                            */
/* at multiples of window_steps of the run's own steps, so a run's result    */
/* does not depend on what else is being served.                             */
/* ------------------------------------------------------------------------ */
typedef struct ecris_server ecris_server;

/* A run to serve: the arguments of ecris_init_fields / ecris_load_ions (host
 * memory; everything is copied at submission) and the convergence rule.
 * Converged (stationary): over two consecutive windows the total extracted
 * current and the currents of the three strongest charge states each change
 * by no more than the larger of rel_tol times the larger of the two values
 * and three standard deviations of the change that the Poisson counts of
 * the two windows allow, with at least min_events extractions in the
 * window. */
typedef struct {
    ecris_geometry geo;
    ecris_bfield bf;
    ecris_grid grid;
    ecris_species sp;
    ecris_mcc mcc;
    size_t n;
    const float* xyzv[6];
    const uint8_t* q;
    double weight;
    uint64_t seed;
    double dt;
    uint32_t window_steps;  /* must divide by the server's steps per tick */
    double rel_tol;
    int64_t min_events;
    uint32_t max_steps;     /* a multiple of window_steps */
    uint32_t ne_windows;    /* 0: the prescribed n_e throughout; k > 0: self-consistent n_e,
                               ecris_update_ne after every k windows of the run's steps */
} ecris_request;

enum { ECRIS_REQ_QUEUED = 0, ECRIS_REQ_RUNNING = 1, ECRIS_REQ_DONE = 2, ECRIS_REQ_FAILED = 3 };

typedef struct {
    int32_t state;          /* ECRIS_REQ_* */
    int32_t converged;      /* 1: rule met before max_steps */
    uint64_t steps;
    double t_submit, t_admit, t_done;   /* s, the server's monotonic clock */
    int32_t qmax;
    int64_t extracted[64];  /* cumulative, per Q */
    int64_t lost[64];
    double current_A[64];   /* over the last window */
    double power_W;
    double ke_lost_eV;
    char error[128];
    double flow_per_s;      /* gas flow over the last window: particles (ions and
                               atoms) out through the aperture per second, times w */
    double power_window_W;  /* power losses (as power_W) over the last window */
} ecris_result;

/* Start a server on `device`: memory budget for resident runs (0: none),
 * steps per tick (the batch advances this many steps between admissions and
 * checks), and the most runs served at once (0: no limit). */
ecris_status ecris_server_create(ecris_server** out, int device, size_t hbm_budget_bytes, uint32_t steps_per_tick,
                                 uint32_t max_active);
/* Stop the loop (runs in flight are abandoned) and release everything. */
void ecris_server_destroy(ecris_server* s);
const char* ecris_server_last_error(const ecris_server* s);
/* Queue a request (thread-safe); *ticket receives its handle.  A request that
 * cannot fit the budget even alone is rejected with ECRIS_ENOMEM. */
ecris_status ecris_server_submit(ecris_server* s, const ecris_request* req, int64_t* ticket);
/* Current state and, once done, the result of a request (thread-safe). */
ecris_status ecris_server_poll(ecris_server* s, int64_t ticket, ecris_result* out);
/* Seconds on the server's clock, and counters: requests queued, running,
 * done; ion-steps advanced since start.  The loop reads a run's tallies one
 * tick after a window boundary while the batch keeps stepping, so a retired
 * run has advanced one tick past the boundary its result belongs to. */
ecris_status ecris_server_stats(ecris_server* s, double* now, int64_t* queued, int64_t* running, int64_t* done,
                                double* ion_steps);
/* How often the request loop has tuned the batch's launch shape (thread-safe).
 * The loop tunes (as ecris_batch_autotune, without the sort-cadence trials,
 * two trial steps a candidate) when runs are resident and their particle
 * count has doubled or halved since the last tuning; the tuner restores every
 * run's state, so no result depends on it. */
ecris_status ecris_server_tunings(ecris_server* s, int64_t* count);

/* Calibration as a served workload (Sec. II: for a given field the model
 * needs two inputs, the macroparticle weight w and the warm-electron
 * temperature T_ew, which are adjusted until the converged plasma's two
 * outputs, the gas flow out of the chamber and the coupled power, meet
 * targets).  A job serves a sequence of runs of `base`, each with the current
 * (w, T_ew) and stepped to convergence (or max_steps) like a request; from
 * the flow F and power P of its last window, with targets Ft and Pt, the
 * next inputs are
 *     w' = w Ft / F,   T_ew' = T_ew (Pt / Ft) / (P / F)
 * (each changed by at most a factor of 4), until both outputs are within
 * tol of the targets or max_iter runs were served.  The first run uses
 * base.weight and base.grid.Te_warm_eV.  At fixed T_ew both outputs are
 * proportional to w; T_ew sets the energy carried out per particle. */
#define ECRIS_CALIB_HISTORY 32
typedef struct {
    ecris_request base;
    double flow_target;     /* particles per second through the aperture */
    double power_target_W;
    double tol;             /* relative, > 0 */
    int32_t max_iter;       /* 1 .. ECRIS_CALIB_HISTORY */
} ecris_calib_request;

typedef struct {
    int32_t state;          /* ECRIS_REQ_*: done when met or after max_iter runs */
    int32_t met;            /* 1: the last run met both targets within tol */
    int32_t iterations;     /* runs finished */
    double weight[ECRIS_CALIB_HISTORY];      /* inputs of run k */
    double Te_warm_eV[ECRIS_CALIB_HISTORY];
    double flow_per_s[ECRIS_CALIB_HISTORY];  /* outputs of run k (last window) */
    double power_W[ECRIS_CALIB_HISTORY];
    uint64_t steps[ECRIS_CALIB_HISTORY];
    char error[128];
} ecris_calib_result;

/* Queue a calibration job (thread-safe; everything is copied); *job receives
 * its handle.  ECRIS_EINVAL for targets <= 0, tol <= 0, max_iter out of
 * range, or a base request ecris_server_submit would reject. */
ecris_status ecris_server_calibrate(ecris_server* s, const ecris_calib_request* req, int64_t* job);
/* State and history of a calibration job (thread-safe). */
ecris_status ecris_server_calib_poll(ecris_server* s, int64_t job, ecris_calib_result* out);

/* Allocation-free Coulomb collision step.  The paper has no counterpart: this
 * is an interface for callers that cannot allocate device memory when they
 * need a collision step -- hosts that reserve all device memory up front and
 * forbid allocation afterwards, plug-ins inside a larger code whose memory
 * manager owns the device, and code that must not let cudaMalloc synchronise
 * the device.  It runs the same Takizawa-Abe pairing and Nanbu scattering as
 * ecris_step (ECRIS_F_COULOMB) on caller-owned device arrays and keeps all its
 * working memory in one fixed-size array that the library holds on every GPU
 * that loads it (about 4.5 MB, until the process exits); it allocates nothing.
 *
 *   n            particles, at most 65536; arrays are indexed by particle id
 *                (the Philox counter word, as in ecris_step)
 *   cell         device, n cell indices (c = (iz*ny + iy)*nx + ix); a particle
 *                takes part when cell < ncells and 1 <= q <= 63
 *   q            device, n charge states
 *   vx, vy, vz   device, n velocities (m/s), updated in place
 *   events       device, n words: ECRIS_EV_COULOMB is OR-ed into the word of
 *                every particle that collided
 *   ncells       1 .. 65536; weight, cell_volume_m3 and lnL_ii give the
 *                density and Coulomb logarithm of Nanbu's s; mass in amu
 *   dt, seed, step  time step (s), Philox key, step index (< 2^30)
 *   cuda_stream  stream to order the work on (NULL: the legacy default stream)
 *   collisions_out  if non-NULL, receives the number of pair collisions and
 *                the call synchronises the stream; otherwise it is asynchronous
 *
 * Larger n or ncells return ECRIS_EINVAL with a message in
 * ecris_last_error(NULL).  Every call shares the one working array: calls whose
 * GPU work overlaps race and must be serialised by the caller.  If they do
 * overlap, a bounded wait inside the call can run out; a call given
 * collisions_out then returns ECRIS_ETIMEOUT (its velocities are not valid),
 * while a call without it returns at once and cannot report this.  The first
 * call on a device sets that device up (a synchronous copy), so make it before
 * any stream capture begins.  That set-up lasts for the life of the process: a
 * device reset (cudaDeviceReset) is not supported. */
ecris_status ecris_coulomb_collide_noalloc(size_t n, const uint32_t* cell, const uint8_t* q, float* vx,
                                           float* vy, float* vz, uint32_t* events, uint32_t ncells,
                                           double mass_amu, double weight, double cell_volume_m3,
                                           double lnL_ii, double dt, uint64_t seed, uint32_t step,
                                           void* cuda_stream, int64_t* collisions_out);

#ifdef __cplusplus
}
#endif

#endif /* ECRIS_H */
