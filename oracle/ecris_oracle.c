/*
 * FP64 CPU oracle of the ECRIS per-macroparticle ion time step.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * timed CPU baseline of the benchmark may load this library.  It shares no
 * code, header, table or constant generator with the CUDA path; both sides
 * take their inputs from the seeded generators and nothing else.
 *
 * The code follows the model of Mironov et al., "Numerical model of Electron
 * Cyclotron Resonance Ion Source" (arXiv:1507.03392), step by step and in the
 * paper's order, in plain loops with no blocking or fusion:
 *   Sec. II (model description): macroparticles, cylinder, mesh, straight
 *     atoms, cosine-law wall re-emission at the gas temperature, extraction
 *     through the round aperture and reinjection at the gas inlet;
 *   Eqs. for B_x, B_y (hexapole added analytically to the solenoid field);
 *   MCC block: ion-ion collisions (Takizawa-Abe pairing, Nanbu angle,
 *     lnL = 10), charge exchange (Q=1 cross section scaled linearly with Q,
 *     Q=2 forbidden, 10 eV release shared equally), electron-ion heating kick
 *     V = V0 + D (R+delta)|R|/|R+delta| with the printed D, and the delta
 *     stencil with R_L, step-wise ionisation from the cell's n_e and T_e;
 *   warm electrons (T_ew) inside the ECR zone, cold (T_ec) outside;
 *   power balance: kinetic + potential energy of lost ions plus 3/2 kT_ew per
 *     lost electron.
 * Readings of points the paper leaves open (synthetic solenoid profile, units
 * of D, Q^2 heating, RNG keying, boundary details) are the ones stated in the
 * repository's design notes; each is repeated at the function that uses it.
 *
 * Functions whose result is pinned by the CPU tests: or_philox (library
 * Philox), or_b0/or_bfield (closed forms, div/curl), or_efield (exact for
 * linear fields), or_lotz_rate (E1 closed form), or_setup_cells and
 * or_cell_delta (delta on a linear ramp, via a prescribed n_e and via the
 * self-consistent n_e of resting ions), or_step (Boris closed forms, mirror invariant, 0-D Markov
 * chains for ionisation and charge exchange, kick moments, wall sampler
 * moments, conservation laws, brute-force deposit), or_nanbu_* (mean cos chi,
 * pair conservation).
 */
#include <math.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdlib.h>
#include <string.h>

#define OR_QE 1.602176634e-19      /* C */
#define OR_AMU 1.66053906660e-27   /* kg */
#define OR_ME 9.1093837015e-31     /* kg */
#define OR_EPS0 8.8541878128e-12   /* F/m */
#define OR_PI 3.14159265358979323846
#define OR_QMAX 64

/* process switches, same bit meaning as the public header */
#define OR_F_PUSH 1u
#define OR_F_IONIZE 2u
#define OR_F_CX 4u
#define OR_F_EIKICK 8u
#define OR_F_COULOMB 16u
#define OR_F_RECYCLE 32u
#define OR_F_ISOHEAT 64u    /* heating kick without the drift bias: delta = 0 */
#define OR_F_DOUBLE 128u    /* double ionisation Q -> Q+2 beside Q -> Q+1 */
#define OR_F_ELASTIC 256u   /* elastic ion-atom scattering, isotropic in the CM frame */
#define OR_F_RECOMB 512u    /* radiative recombination Q -> Q-1 */

/* per-particle event bits of one step */
#define OR_EV_WALL 1u
#define OR_EV_EXTRACT 2u
#define OR_EV_IONIZE 4u
#define OR_EV_CX 8u
#define OR_EV_COULOMB 16u
#define OR_EV_ELASTIC 32u
#define OR_EV_RECOMB 64u

/* guard bits: outcomes within rounding distance of a decision surface */
#define OR_G_CELL 1u
#define OR_G_BOUNDARY 2u
#define OR_G_IONIZE 4u
#define OR_G_CX 8u
#define OR_G_CELLREC 16u   /* near a cell face whose other side has different electron data */

typedef struct {
    double R0, L, r_ap, inlet[3];
    double B_inj, B_min, B_ext, B_hex, B_ecr;
    int32_t nx, ny, nz, qmax;
    double mass_amu;
    double Te_warm, Te_cold;         /* eV */
    double n0_m3, T0_eV, sigma1_m2, E_cx_eV, lnL_ii, lnL_ei;
    int32_t ei_charge_power;
    uint32_t flags;
    double weight;
    uint64_t seed;
    double dt;
    double T_refl_eV;                /* re-emission temperature of ions neutralised at a wall (0: T0) */
    double sigma_el_m2;              /* elastic ion-atom cross section of Q = 1 (scaled by Q) */
    double k2_factor;                /* double-ionisation rate factor */
    double k3_factor;                /* triple-ionisation rate factor (0: off) */
    int32_t ax_n;                    /* on-axis B0 table: samples at z_k = k L/(ax_n - 1); 0: mirror */
    const double *ax_y;              /* B0(z_k), T */
    const double *ax_M;              /* the natural cubic spline's B0''(z_k) (or_axial_setup) */
} or_params;

typedef struct {
    int64_t extracted[OR_QMAX];
    int64_t lost[OR_QMAX];
    double ke_lost_eV;   /* kinetic energy of ions (Q>=1) leaving the chamber */
    int64_t coulomb_pairs;
    double r_ext_sum[OR_QMAX];   /* radius at the aperture plane summed over extracted particles (m) */
} or_tally;

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).  Ten rounds of two     */
/* 32x32->64 multiplies with the published multipliers; the key is bumped by */
/* the published Weyl constants between rounds.                              */
/* ------------------------------------------------------------------------ */
void or_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t pa = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t pb = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi_a = (uint32_t)(pa >> 32), lo_a = (uint32_t)pa;
        uint32_t hi_b = (uint32_t)(pb >> 32), lo_b = (uint32_t)pb;
        uint32_t n0 = hi_b ^ c1 ^ k0;
        uint32_t n1 = lo_b;
        uint32_t n2 = hi_a ^ c3 ^ k1;
        uint32_t n3 = lo_a;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* The method's random words for particle `pid` at step `step`, stream s:
 * counter (pid, 0, 4*step + s, 0), key (seed low, seed high).
 * Streams: 0 = MCC (ionisation, CX, two kick words), 1 = Coulomb pairing key
 * and angles, 2 = wall re-emission / reinjection, 3 = charge-exchange
 * product velocity. */
static void or_words(uint64_t seed, uint32_t pid, uint32_t step, uint32_t s, uint32_t w[4])
{
    uint32_t ctr[4] = {pid, 0u, step * 4u + s, 0u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    or_philox(ctr, key, w);
}

/* uniform in (0, 1], the top 24 bits of a word plus one, times 2^-24 */
static double or_unit(uint32_t w) { return ((double)(w >> 8) + 1.0) * (1.0 / 16777216.0); }

/* decision threshold: an event fires when the word is below floor(p 2^32) */
static double or_threshold(double p) { return p * 4294967296.0; }

/* ------------------------------------------------------------------------ */
/* Magnetic field.  The solenoid maps (Poisson-Superfish) are not available; */
/* the on-axis profile B0(z) is a synthetic mirror through the three printed */
/* extremes: B_inj at z=0 (injection side), B_min at z_m, B_ext at z=L,      */
/* raised-cosine halves joined with continuous B0''.  Off axis the paraxial  */
/* expansion B_r = -(r/2) B0', B_z = B0 - (r^2/4) B0'' is used.  The         */
/* hexapole is added as printed: B_x += B_H sin(2 theta) R^2/R0^2,           */
/* B_y += B_H cos(2 theta) R^2/R0^2.                                          */
/* ------------------------------------------------------------------------ */
double or_zmin(const or_params *p)
{
    double ratio = sqrt((p->B_ext - p->B_min) / (p->B_inj - p->B_min));
    return p->L / (1.0 + ratio);
}

/* Natural cubic spline through n samples y_k at z_k = k h (h = L/(n-1)):
 * its second derivatives M_k solve M_0 = M_{n-1} = 0 and
 * M_{k-1} + 4 M_k + M_{k+1} = 6 (y_{k+1} - 2 y_k + y_{k-1}) / h^2, by
 * forward elimination and back substitution (Thomas algorithm). */
void or_axial_setup(int32_t n, double L, const double *y, double *M)
{
    double h = L / (n - 1);
    double *c = (double *)malloc((size_t)n * sizeof(double));
    double *d = (double *)malloc((size_t)n * sizeof(double));
    M[0] = 0.0;
    M[n - 1] = 0.0;
    /* unknowns M_1 .. M_{n-2}: diagonal 4, off-diagonals 1 */
    for (int k = 1; k <= n - 2; ++k) {
        double rhs = 6.0 * (y[k + 1] - 2.0 * y[k] + y[k - 1]) / (h * h);
        double diag = 4.0 - (k > 1 ? c[k - 1] : 0.0);
        c[k] = 1.0 / diag;
        d[k] = (rhs - (k > 1 ? d[k - 1] : 0.0)) / diag;
    }
    for (int k = n - 2; k >= 1; --k) M[k] = d[k] - c[k] * (k < n - 2 ? M[k + 1] : 0.0);
    free(c);
    free(d);
}

/* B0, B0', B0'' of the spline on the segment holding z (clamped to the ends):
 * with t = (z - z_k)/h, B0 = (1-t) y_k + t y_{k+1} + h^2/6 [((1-t)^3 - (1-t)) M_k
 * + (t^3 - t) M_{k+1}] and its derivatives in z. */
static void or_b0_axial(const or_params *p, double z, double out[3])
{
    int n = p->ax_n;
    double h = p->L / (n - 1);
    int k = (int)floor(z / h);
    if (k < 0) k = 0;
    if (k > n - 2) k = n - 2;
    double t = (z - k * h) / h, u = 1.0 - t;
    const double *y = p->ax_y, *M = p->ax_M;
    out[0] = u * y[k] + t * y[k + 1] + h * h / 6.0 * ((u * u * u - u) * M[k] + (t * t * t - t) * M[k + 1]);
    out[1] = (y[k + 1] - y[k]) / h + h / 6.0 * (-(3.0 * u * u - 1.0) * M[k] + (3.0 * t * t - 1.0) * M[k + 1]);
    out[2] = u * M[k] + t * M[k + 1];
}

void or_b0(const or_params *p, double z, double out[3])
{
    if (p->ax_n > 0) {
        or_b0_axial(p, z, out);
        return;
    }
    double zm = or_zmin(p);
    if (z <= zm) {
        double a = 0.5 * (p->B_inj - p->B_min), k = OR_PI / zm;
        out[0] = p->B_min + a * (1.0 + cos(k * z));
        out[1] = -a * k * sin(k * z);
        out[2] = -a * k * k * cos(k * z);
    } else {
        double a = 0.5 * (p->B_ext - p->B_min), k = OR_PI / (p->L - zm);
        out[0] = p->B_min + a * (1.0 - cos(k * (z - zm)));
        out[1] = a * k * sin(k * (z - zm));
        out[2] = a * k * k * cos(k * (z - zm));
    }
}

void or_bfield(const or_params *p, double x, double y, double z, double B[3])
{
    double b0[3];
    or_b0(p, z, b0);
    double r2 = x * x + y * y;
    double R = sqrt(r2);
    /* solenoid, paraxial: B_r cos(theta) = -(x/2) B0', B_r sin(theta) = -(y/2) B0' */
    double Bx = -0.5 * x * b0[1];
    double By = -0.5 * y * b0[1];
    double Bz = b0[0] - 0.25 * r2 * b0[2];
    /* hexapole as printed, with theta the polar angle */
    if (R > 0.0) {
        double th = atan2(y, x);
        double s = p->B_hex * R * R / (p->R0 * p->R0);
        Bx += s * sin(2.0 * th);
        By += s * cos(2.0 * th);
    }
    B[0] = Bx; B[1] = By; B[2] = Bz;
}

/* ------------------------------------------------------------------------ */
/* Mesh: nx x ny x nz cells over [-R0,R0]^2 x [0,L]; cell index             */
/* c = (iz*ny + iy)*nx + ix.                                                 */
/* ------------------------------------------------------------------------ */
static double or_dx(const or_params *p) { return 2.0 * p->R0 / p->nx; }
static double or_dy(const or_params *p) { return 2.0 * p->R0 / p->ny; }
static double or_dz(const or_params *p) { return p->L / p->nz; }

static int or_clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* nearest-grid-point cell of a position: the cell whose plasma parameters act on the particle */
static int64_t or_cell(const or_params *p, double x, double y, double z, uint32_t *guard)
{
    double gx = (x + p->R0) / or_dx(p), gy = (y + p->R0) / or_dy(p), gz = z / or_dz(p);
    const double tol = 1e-4; /* cell units */
    if (guard) {
        if (fabs(gx - floor(gx + 0.5)) < tol || fabs(gy - floor(gy + 0.5)) < tol ||
            fabs(gz - floor(gz + 0.5)) < tol)
            *guard |= OR_G_CELL;
    }
    int ix = or_clampi((int)floor(gx), 0, p->nx - 1);
    int iy = or_clampi((int)floor(gy), 0, p->ny - 1);
    int iz = or_clampi((int)floor(gz), 0, p->nz - 1);
    return ((int64_t)iz * p->ny + iy) * p->nx + ix;
}

/* 1 if a flip of the particle's cell across a face it lies within the guard
 * distance of could change its outcome this step: the ionisation decision
 * (word w0 against the probability from the other cell's n_e and zone) or,
 * for an ion, the heating kick (the other cell's n_e, zone or delta). */
static int or_ion_outcome(const or_params *p, double ne_c, int zc, const double *rates, const double *rates2,
                          const double *ratesr, int Q, uint32_t w0, int *near);

static int or_cell_record_guard(const or_params *p, double x, double y, double z, int64_t c,
                                const double *ne, const int32_t *zone, const double *dlx,
                                const double *dly, const double *rates, const double *rates2,
                                const double *ratesr, int q_before, int q_after, uint32_t w0)
{
    const double tol = 1e-4;
    double g[3] = {(x + p->R0) / or_dx(p), (y + p->R0) / or_dy(p), z / or_dz(p)};
    int n[3] = {p->nx, p->ny, p->nz};
    int64_t stride[3] = {1, p->nx, (int64_t)p->nx * p->ny};
    int idx[3] = {(int)(c % p->nx), (int)((c / p->nx) % p->ny), (int)(c / ((int64_t)p->nx * p->ny))};
    for (int k = 0; k < 3; ++k) {
        double r = g[k] - floor(g[k] + 0.5);
        if (fabs(r) >= tol) continue;
        /* the nearest face is below the cell when g sits just above an integer */
        int other = (g[k] - idx[k] < 0.5) ? idx[k] - 1 : idx[k] + 1;
        if (other < 0 || other >= n[k]) continue;
        int64_t c2 = c + (other - idx[k]) * stride[k];
        if ((((p->flags & OR_F_IONIZE) && q_before < p->qmax) || ((p->flags & OR_F_RECOMB) && q_before >= 1)) &&
            or_ion_outcome(p, ne[c], zone[c], rates, rates2, ratesr, q_before, w0, NULL) !=
                or_ion_outcome(p, ne[c2], zone[c2], rates, rates2, ratesr, q_before, w0, NULL))
            return 1;
        if ((p->flags & OR_F_EIKICK) && q_after >= 1 &&
            (ne[c2] != ne[c] || zone[c2] != zone[c] || dlx[c2] != dlx[c] || dly[c2] != dly[c]))
            return 1;
    }
    return 0;
}

/* E at a position: trilinear interpolation between cell centres of the
 * cell-centred grid E[3*c + k]; positions within half a cell of an outer face
 * take the face cell's value along that axis. */
static void or_axis(double g, int n, int *i0, double *f)
{
    double gc = g - 0.5;
    int i = (int)floor(gc);
    if (i < 0) { *i0 = 0; *f = 0.0; return; }
    if (i > n - 2) { *i0 = n - 2; *f = 1.0; return; }
    *i0 = i; *f = gc - i;
}

void or_efield(const or_params *p, const double *E, double x, double y, double z, double out[3])
{
    int ix, iy, iz;
    double fx, fy, fz;
    or_axis((x + p->R0) / or_dx(p), p->nx, &ix, &fx);
    or_axis((y + p->R0) / or_dy(p), p->ny, &iy, &fy);
    or_axis(z / or_dz(p), p->nz, &iz, &fz);
    out[0] = out[1] = out[2] = 0.0;
    for (int cz = 0; cz < 2; ++cz)
        for (int cy = 0; cy < 2; ++cy)
            for (int cx = 0; cx < 2; ++cx) {
                double w = (cx ? fx : 1.0 - fx) * (cy ? fy : 1.0 - fy) * (cz ? fz : 1.0 - fz);
                int64_t c = ((int64_t)(iz + cz) * p->ny + (iy + cy)) * p->nx + (ix + cx);
                for (int k = 0; k < 3; ++k) out[k] += w * E[3 * c + k];
            }
}

/* ------------------------------------------------------------------------ */
/* Ionisation rates.  The datasets [20-23] are not available; the rate of    */
/* Q -> Q+1 is the Maxwellian average (the paper's Maxwellian EEDF) of the   */
/* single-term Lotz cross section sigma(E) = a q ln(E/P) / (E P), a = 4.5e-14 */
/* cm^2 eV^2, computed here by direct quadrature:                            */
/*   k = sqrt(8/(pi m_e)) (kT)^-3/2 Int_P^inf sigma(E) E exp(-E/kT) dE.       */
/* Returns m^3/s.                                                            */
/* ------------------------------------------------------------------------ */
double or_lotz_rate(double P_eV, int q_outer, double Te_eV)
{
    const double a = 4.5e-14 * 1e-4; /* m^2 eV^2 */
    /* substitute E = P + Te t; integrand sigma(E) E exp(-E/Te) Te dt */
    const int n = 200000;          /* Simpson intervals (even) */
    const double tmax = 80.0;
    double h = tmax / n, sum = 0.0;
    for (int i = 0; i <= n; ++i) {
        double t = i * h;
        double E = P_eV + Te_eV * t;
        double f = a * q_outer * log(E / P_eV) / P_eV * exp(-t);
        double w = (i == 0 || i == n) ? 1.0 : ((i & 1) ? 4.0 : 2.0);
        sum += w * f;
    }
    double integral = sum * h / 3.0 * Te_eV * exp(-P_eV / Te_eV); /* m^2 eV^2 */
    double kT = Te_eV * OR_QE;                                     /* J */
    double vfac = sqrt(8.0 / (OR_PI * OR_ME));                     /* (J/kg)^1/2 per J^1/2 */
    /* integral is in m^2 eV^2; convert eV^2 -> J^2, then k = vfac kT^-3/2 integral */
    return vfac * pow(kT, -1.5) * integral * OR_QE * OR_QE;
}

/* rates[zone*qmax + Q], zone 0 = cold electrons, 1 = warm */
void or_build_rates(const or_params *p, const double *ip_eV, const int32_t *n_outer, double *rates)
{
    for (int zone = 0; zone < 2; ++zone) {
        double Te = zone ? p->Te_warm : p->Te_cold;
        for (int q = 0; q < p->qmax; ++q)
            rates[zone * p->qmax + q] = or_lotz_rate(ip_eV[q], n_outer[q], Te);
    }
}

/* Multiple ionisation (Sec. II; the fit of [22] for two electrons and the
 * scaling of [23] for three are not available).  Double, Q -> Q+2:
 * k2_factor times the Lotz-Maxwellian rate with the threshold P_Q + P_{Q+1}
 * (both electrons removed) and q_Q outer electrons, in rates2[zone*qmax + Q],
 * zero for Q = qmax - 1.  Triple, Q -> Q+3: k3_factor times the same with
 * the threshold P_Q + P_{Q+1} + P_{Q+2}, in rates2[2*qmax + zone*qmax + Q],
 * zero for Q >= qmax - 2.  Four or more electrons are left out (the paper
 * finds the processes beyond double ionisation minor contributors). */
void or_build_rates2(const or_params *p, const double *ip_eV, const int32_t *n_outer, double *rates2)
{
    for (int zone = 0; zone < 2; ++zone) {
        double Te = zone ? p->Te_warm : p->Te_cold;
        for (int q = 0; q < p->qmax; ++q) {
            rates2[zone * p->qmax + q] =
                q + 1 < p->qmax ? p->k2_factor * or_lotz_rate(ip_eV[q] + ip_eV[q + 1], n_outer[q], Te) : 0.0;
            rates2[2 * p->qmax + zone * p->qmax + q] =
                q + 2 < p->qmax && p->k3_factor > 0.0
                    ? p->k3_factor * or_lotz_rate(ip_eV[q] + ip_eV[q + 1] + ip_eV[q + 2], n_outer[q], Te)
                    : 0.0;
        }
    }
}

/* Radiative recombination Q -> Q-1 (Sec. II; the datasets [21] are not
 * available): Seaton's hydrogenic rate for an ion of charge Z = Q,
 * alpha = 5.197e-14 Z lambda^1/2 (0.4288 + 0.5 ln lambda + 0.469 lambda^-1/3)
 * cm^3/s with lambda = 157890 Z^2 / T(K), T = T_e.  ratesr[zone*(qmax+1) + Q],
 * zero for atoms. */
double or_recomb_rate(int Z, double Te_eV)
{
    double TK = Te_eV * 11604.518;
    double lam = 157890.0 * Z * Z / TK;
    return 5.197e-14 * Z * sqrt(lam) * (0.4288 + 0.5 * log(lam) + 0.469 * pow(lam, -1.0 / 3.0)) * 1e-6;
}

void or_build_rates_rec(const or_params *p, double *ratesr)
{
    for (int zone = 0; zone < 2; ++zone) {
        double Te = zone ? p->Te_warm : p->Te_cold;
        for (int q = 0; q <= p->qmax; ++q)
            ratesr[zone * (p->qmax + 1) + q] = q >= 1 ? or_recomb_rate(q, Te) : 0.0;
    }
}

static int or_near(double w0, double t) { return fabs(w0 - t) < 1e-5 * t + 2.0; }

/* Outcome of the ionisation word w0 in a cell: 0 none, 1 single, 2 double,
 * 3 triple, -1 recombination.
 * One step's probability of any of these is p = 1 - exp(-n_e k dt) with
 * k = k1 + k2 + k3 + kr (the processes switched on); it is shared in
 * proportion to the rates, so w0 below p k1/k ionises once, below
 * p (k1+k2)/k twice, below p (k1+k2+k3)/k three times, and below p
 * recombines.  *near is set when w0 lies within rounding distance of any of
 * the thresholds. */
static int or_ion_outcome(const or_params *p, double ne_c, int zc, const double *rates, const double *rates2,
                          const double *ratesr, int Q, uint32_t w0, int *near)
{
    const int rec = ratesr && (p->flags & OR_F_RECOMB);
    const int ion = rec ? ((p->flags & OR_F_IONIZE) && Q < p->qmax) : 1;
    const int multi = ion && rates2 && (p->flags & OR_F_DOUBLE);
    double k1 = ion ? rates[zc * p->qmax + Q] : 0.0;
    double k2 = multi ? rates2[zc * p->qmax + Q] : 0.0;
    double k3 = multi ? rates2[2 * p->qmax + zc * p->qmax + Q] : 0.0;
    double kr = rec ? ratesr[zc * (p->qmax + 1) + Q] : 0.0;
    double w = (double)w0;
    if (!rec && k2 <= 0.0 && k3 <= 0.0) {
        double thr = or_threshold(-expm1(-ne_c * k1 * p->dt));
        if (near && or_near(w, thr)) *near = 1;
        return w < floor(thr) ? 1 : 0;
    }
    double k = k1 + k2 + k3 + kr;
    if (k <= 0.0) return 0;
    double pt = -expm1(-ne_c * k * p->dt);
    double t = or_threshold(pt), t1 = or_threshold(pt * (k1 / k)), t2 = or_threshold(pt * ((k1 + k2) / k)),
           t3 = or_threshold(pt * ((k1 + k2 + k3) / k));
    if (near && (or_near(w, t) || or_near(w, t1) || or_near(w, t2) || or_near(w, t3))) *near = 1;
    if (w < floor(t1)) return 1;
    if (w < floor(t2)) return 2;
    if (w < floor(t3)) return 3;
    return w < floor(t) ? -1 : 0;
}

/* ------------------------------------------------------------------------ */
/* Per-cell electron data.  A cell is in the ECR zone (warm electrons) when */
/* |B| at its centre is below B_ECR.  n_e there is the per-cell input (or   */
/* the scalar ne_in), ne_out outside; inputs in cm^-3, stored in m^-3.       */
/* delta (x, y components; z = 0) follows the printed 3x3 stencil scaled by  */
/* R_L = 2.38e-6 sqrt(T_e) / (B dX); neighbours outside the mesh take the    */
/* edge cell's value and a cell with n_e = 0 gets delta = 0.                 */
/* ------------------------------------------------------------------------ */
void or_cell_delta(const or_params *p, const double *ne, const int32_t *zone, const double *Bmag,
                   double *dlx, double *dly);

void or_setup_cells(const or_params *p, const float *ne_in_cells, double ne_in_cm3,
                    double ne_out_cm3, double *ne, int32_t *zone, double *Bmag,
                    double *dlx, double *dly)
{
    int nx = p->nx, ny = p->ny, nz = p->nz;
    double dx = or_dx(p), dy = or_dy(p), dz = or_dz(p);
    for (int iz = 0; iz < nz; ++iz)
        for (int iy = 0; iy < ny; ++iy)
            for (int ix = 0; ix < nx; ++ix) {
                int64_t c = ((int64_t)iz * ny + iy) * nx + ix;
                double B[3];
                or_bfield(p, -p->R0 + (ix + 0.5) * dx, -p->R0 + (iy + 0.5) * dy, (iz + 0.5) * dz, B);
                double b = sqrt(B[0] * B[0] + B[1] * B[1] + B[2] * B[2]);
                Bmag[c] = b;
                zone[c] = b < p->B_ecr ? 1 : 0;
                double nin = ne_in_cells ? (double)ne_in_cells[c] : ne_in_cm3;
                ne[c] = (zone[c] ? nin : ne_out_cm3) * 1e6;
            }
    or_cell_delta(p, ne, zone, Bmag, dlx, dly);
}

/* delta of every cell from n_e (m^-3), the zone flags and |B|: the stencil   */
/* and R_L above.  Called at setup and again whenever n_e is replaced by the */
/* ions' charge density (Sec. II, charge neutrality).                         */
void or_cell_delta(const or_params *p, const double *ne, const int32_t *zone, const double *Bmag,
                   double *dlx, double *dly)
{
    int nx = p->nx, ny = p->ny, nz = p->nz;
    double dx = or_dx(p);
    if (p->flags & OR_F_ISOHEAT) {
        /* isotropic heating (Sec. IV): the kick without the drift bias */
        for (int64_t c = 0; c < (int64_t)nx * ny * nz; ++c) { dlx[c] = 0.0; dly[c] = 0.0; }
        return;
    }
    for (int iz = 0; iz < nz; ++iz)
        for (int iy = 0; iy < ny; ++iy)
            for (int ix = 0; ix < nx; ++ix) {
                int64_t c = ((int64_t)iz * ny + iy) * nx + ix;
#define NE(i, j) ne[((int64_t)iz * ny + or_clampi(j, 0, ny - 1)) * nx + or_clampi(i, 0, nx - 1)]
                double n0 = ne[c];
                if (n0 <= 0.0) { dlx[c] = 0.0; dly[c] = 0.0; continue; }
                double Te = zone[c] ? p->Te_warm : p->Te_cold;
                double RL = 2.38e-6 * sqrt(Te) / (Bmag[c] * dx);
                double sx = -NE(ix, iy + 1) + NE(ix, iy - 1) +
                            0.5 * (-NE(ix - 1, iy + 1) - NE(ix + 1, iy + 1) +
                                   NE(ix + 1, iy - 1) + NE(ix - 1, iy - 1));
                double sy = -NE(ix - 1, iy) + NE(ix + 1, iy) +
                            0.5 * (-NE(ix - 1, iy + 1) + NE(ix + 1, iy + 1) +
                                   NE(ix + 1, iy - 1) - NE(ix - 1, iy - 1));
#undef NE
                dlx[c] = -RL / n0 * sx;
                dly[c] = -RL / n0 * sy;
            }
}

/* Threads of the particle loop (the timed CPU baseline runs on all cores and
 * on one); returns the count in effect. */
int or_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Boris rotation (Boris 1970): half electric kick, magnetic rotation by     */
/* t = (qB/m) dt/2, s = 2t/(1+t^2), second half kick.                        */
/* ------------------------------------------------------------------------ */
static void or_cross(const double a[3], const double b[3], double o[3])
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

void or_boris(double qm, const double E[3], const double B[3], double dt, double v[3])
{
    double vm[3], t[3], s[3], vp[3], c[3];
    for (int k = 0; k < 3; ++k) { vm[k] = v[k] + qm * E[k] * 0.5 * dt; t[k] = qm * B[k] * 0.5 * dt; }
    double t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
    for (int k = 0; k < 3; ++k) s[k] = 2.0 * t[k] / (1.0 + t2);
    or_cross(vm, t, c);
    for (int k = 0; k < 3; ++k) vp[k] = vm[k] + c[k];
    or_cross(vp, s, c);
    for (int k = 0; k < 3; ++k) v[k] = vm[k] + c[k] + qm * E[k] * 0.5 * dt;
}

/* ------------------------------------------------------------------------ */
/* Cosine-law re-emission with full accommodation at temperature T0: normal  */
/* speed flux-weighted Maxwellian (v_n = sigma sqrt(-2 ln U)), tangential    */
/* components Maxwellian (one Box-Muller pair), sigma^2 = kT0/M.  Uses the   */
/* stream-2 words w[0] (normal), w[1], w[2] (tangential).                    */
/* ------------------------------------------------------------------------ */
void or_emit(double sigma, const double n[3], const double e1[3], const double e2[3],
             const uint32_t w[4], double v[3])
{
    double vn = sigma * sqrt(-2.0 * log(or_unit(w[0])));
    double rt = sigma * sqrt(-2.0 * log(or_unit(w[1])));
    double th = 2.0 * OR_PI * or_unit(w[2]);
    double t1 = rt * cos(th), t2 = rt * sin(th);
    for (int k = 0; k < 3; ++k) v[k] = vn * n[k] + t1 * e1[k] + t2 * e2[k];
}

/* ------------------------------------------------------------------------ */
/* Takizawa-Abe pairing with Nanbu's scattering angle.                       */
/* ------------------------------------------------------------------------ */
/* A(s) from coth(A) - 1/A = exp(-s): bisection in A on a bracket, then the
 * large-A form 1/(1 - exp(-s)) when the root sits beyond double precision's
 * reach of coth. */
double or_nanbu_A(double s)
{
    double target = exp(-s);
    if (s < 1e-3) return 1.0 / (-expm1(-s)) ; /* coth(A) = 1 to double precision */
    double lo = 1e-12, hi = 2.0 / (-expm1(-s)) + 10.0;
    for (int it = 0; it < 80; ++it) {
        double mid = 0.5 * (lo + hi);
        double f = 1.0 / tanh(mid) - 1.0 / mid - target;
        if (f < 0.0) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

/* cos(chi) for uniform U in (0,1]: Nanbu's cos chi = A^-1 ln(e^-A + 2U sinh A),
 * written as 1 + A^-1 ln(U + (1-U) e^-2A) to stay finite for large A; for
 * s > 6 the angle is isotropic, cos chi = 2U - 1. */
double or_nanbu_cos(double s, double U)
{
    if (s > 6.0) return 2.0 * U - 1.0;
    double A = or_nanbu_A(s);
    double c = 1.0 + log(U + (1.0 - U) * exp(-2.0 * A)) / A;
    if (c > 1.0) c = 1.0;
    if (c < -1.0) c = -1.0;
    return c;
}

/* Rotate the relative velocity of an equal-mass pair by (chi, eps) and share
 * the change equally: va += dg/2, vb -= dg/2. */
void or_scatter_pair(double *va, double *vb, double cos_chi, double eps)
{
    double g[3] = {va[0] - vb[0], va[1] - vb[1], va[2] - vb[2]};
    double gm = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    if (gm == 0.0) return;
    double gp = sqrt(g[1] * g[1] + g[2] * g[2]);
    double sin_chi = sqrt(fmax(0.0, 1.0 - cos_chi * cos_chi));
    double ce = cos(eps), se = sin(eps);
    double h[3];
    if (gp > 0.0) {
        h[0] = gp * ce;
        h[1] = -(g[0] * g[1] * ce + gm * g[2] * se) / gp;
        h[2] = -(g[0] * g[2] * ce - gm * g[1] * se) / gp;
    } else {
        h[0] = 0.0; h[1] = gm * ce; h[2] = gm * se;
    }
    for (int k = 0; k < 3; ++k) {
        double dg = g[k] * (cos_chi - 1.0) + h[k] * sin_chi;
        va[k] += 0.5 * dg;
        vb[k] -= 0.5 * dg;
    }
}

/* s of one collision between charges Qa, Qb (same mass M): Nanbu's
 * s = (lnL/4pi) (Qa Qb e^2 / (eps0 mu))^2 n g^-3 dt, mu = M/2. */
double or_nanbu_s(double lnL, double Qa, double Qb, double mass_kg, double n_m3, double g, double dt)
{
    double mu = 0.5 * mass_kg;
    double k = Qa * Qb * OR_QE * OR_QE / (OR_EPS0 * mu);
    return lnL / (4.0 * OR_PI) * k * k * n_m3 / (g * g * g) * dt;
}

typedef struct { uint32_t hash; uint32_t pid; } or_key;

static int or_key_cmp(const void *a, const void *b)
{
    const or_key *x = (const or_key *)a, *y = (const or_key *)b;
    if (x->hash != y->hash) return x->hash < y->hash ? -1 : 1;
    if (x->pid != y->pid) return x->pid < y->pid ? -1 : 1;
    return 0;
}

/* One collision of the pair (a, b) over time dt_c, using the stream-1 words
 * of particle `first`: w[1] -> cos chi, w[2] -> azimuth eps. */
static void or_collide(const or_params *p, double *vx, double *vy, double *vz, const int32_t *q,
                       uint32_t a, uint32_t b, double n_m3, double dt_c, uint32_t step,
                       uint32_t first)
{
    double va[3] = {vx[a], vy[a], vz[a]}, vb[3] = {vx[b], vy[b], vz[b]};
    double g = sqrt((va[0] - vb[0]) * (va[0] - vb[0]) + (va[1] - vb[1]) * (va[1] - vb[1]) +
                    (va[2] - vb[2]) * (va[2] - vb[2]));
    if (g <= 0.0) return;
    uint32_t w[4];
    or_words(p->seed, first, step, 1, w);
    double s = or_nanbu_s(p->lnL_ii, q[a], q[b], p->mass_amu * OR_AMU, n_m3, g, dt_c);
    double cchi = or_nanbu_cos(s, or_unit(w[1]));
    double eps = 2.0 * OR_PI * or_unit(w[2]);
    or_scatter_pair(va, vb, cchi, eps);
    vx[a] = va[0]; vy[a] = va[1]; vz[a] = va[2];
    vx[b] = vb[0]; vy[b] = vb[1]; vz[b] = vb[2];
}

/* Coulomb step over all cells.  `part` lists the particles taking part (ions
 * that stayed inside this step) with their cell.  Inside a cell the ions are
 * ordered by (stream-1 word 0, pid); consecutive ions pair up; with an odd
 * count the first three collide pairwise (0,1), (1,2), (2,0) over dt/2 each. */
static void or_coulomb(const or_params *p, int64_t n, const int64_t *cell, const uint8_t *part,
                       double *vx, double *vy, double *vz, const int32_t *q, uint32_t step,
                       double dt, uint8_t *events, or_tally *t)
{
    int64_t nc = (int64_t)p->nx * p->ny * p->nz;
    int64_t *cnt = (int64_t *)calloc((size_t)nc + 1, sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) if (part[i]) cnt[cell[i] + 1]++;
    for (int64_t c = 0; c < nc; ++c) cnt[c + 1] += cnt[c];
    int64_t total = cnt[nc];
    or_key *keys = (or_key *)malloc((size_t)(total > 0 ? total : 1) * sizeof(or_key));
    int64_t *fill = (int64_t *)malloc((size_t)nc * sizeof(int64_t));
    for (int64_t c = 0; c < nc; ++c) fill[c] = cnt[c];
    /* each participant's pairing word (independent per particle) */
    uint32_t *hash = (uint32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(uint32_t));
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        if (!part[i]) continue;
        uint32_t w[4];
        or_words(p->seed, (uint32_t)i, step, 1, w);
        hash[i] = w[0];
    }
    for (int64_t i = 0; i < n; ++i) {
        if (!part[i]) continue;
        or_key k = {hash[i], (uint32_t)i};
        keys[fill[cell[i]]++] = k;
    }
    double vcell = or_dx(p) * or_dy(p) * or_dz(p);
    /* the cells are independent: each collides only its own ions */
    int64_t pairs = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : pairs)
    for (int64_t c = 0; c < nc; ++c) {
        int64_t m = cnt[c + 1] - cnt[c];
        if (m < 2) continue;
        or_key *k = keys + cnt[c];
        qsort(k, (size_t)m, sizeof(or_key), or_key_cmp);
        double n_m3 = p->weight * (double)m / vcell;
        int64_t start = 0;
        if (m & 1) {
            or_collide(p, vx, vy, vz, q, k[0].pid, k[1].pid, n_m3, 0.5 * dt, step, k[0].pid);
            or_collide(p, vx, vy, vz, q, k[1].pid, k[2].pid, n_m3, 0.5 * dt, step, k[1].pid);
            or_collide(p, vx, vy, vz, q, k[2].pid, k[0].pid, n_m3, 0.5 * dt, step, k[2].pid);
            for (int j = 0; j < 3; ++j) events[k[j].pid] |= OR_EV_COULOMB;
            pairs += 3;
            start = 3;
        }
        for (int64_t j = start; j + 1 < m; j += 2) {
            or_collide(p, vx, vy, vz, q, k[j].pid, k[j + 1].pid, n_m3, dt, step, k[j].pid);
            events[k[j].pid] |= OR_EV_COULOMB;
            events[k[j + 1].pid] |= OR_EV_COULOMB;
            pairs += 1;
        }
    }
    t->coulomb_pairs += pairs;
    free(cnt); free(keys); free(fill); free(hash);
}

/* ------------------------------------------------------------------------ */
/* One time step for particles 0..n-1 of one run, in the paper's order:      */
/*  1. push (Boris for ions in B + interpolated E; atoms straight),          */
/*  2. boundary test on the new position (wall, or aperture at z = L),       */
/*  3. MCC for particles that stayed: ionisation, charge exchange, e-i kick, */
/*     then ion-ion Coulomb over all cells,                                  */
/*  4. wall / aperture bookkeeping for particles that left,                  */
/*  5. NGP deposition of count and charge at the final position.             */
/* rates: from or_build_rates.  cell arrays: from or_setup_cells.  E: 3*Nc.   */
/* status[i] bit 0 = frozen (left with recycling off).                       */
/* events/guard: per-particle outputs of this step.                          */
/* dep_count/dep_charge: Nc accumulators (may be NULL).                      */
/* ------------------------------------------------------------------------ */
#define OR_LEAVE_NONE 0
#define OR_LEAVE_RADIAL 1
#define OR_LEAVE_Z0 2
#define OR_LEAVE_ZL 3
#define OR_LEAVE_APERTURE 4

void or_step(const or_params *p, const double *rates, const double *rates2, const double *ratesr,
             const double *ne, const int32_t *zone,
             const double *dlx, const double *dly, const double *E, int64_t n, double *x,
             double *y, double *z, double *vx, double *vy, double *vz, int32_t *q,
             uint32_t *status, uint32_t step, uint8_t *events, uint8_t *guard, or_tally *t,
             int64_t *dep_count, int64_t *dep_charge)
{
    const double dt = p->dt;
    const double M = p->mass_amu * OR_AMU;
    const double gband = 1e-4 * fmin(or_dx(p), or_dz(p)); /* metres */
    const double eps_wall = 1e-6 * p->L;
    const double sig0 = sqrt(p->T0_eV * OR_QE / M);
    /* ions neutralised at a wall come back at T_refl (Sec. III.C, warm
     * reflected atoms); atoms hitting a wall and reinjected gas at T0 */
    const double sig_refl = p->T_refl_eV > 0.0 ? sqrt(p->T_refl_eV * OR_QE / M) : sig0;
    int64_t *cell = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    uint8_t *leave = (uint8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
    uint8_t *part = (uint8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
    double *xc = (double *)malloc((size_t)(n > 0 ? n : 1) * 3 * sizeof(double));
    int32_t *qleave = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));

    /* phase 1: push, boundary test, MCC (single-particle processes; each
     * iteration touches only particle i, so the loop may run in parallel) */
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        events[i] = 0; guard[i] = 0; cell[i] = -1;
        if (status[i] & 1u) continue;
        double v[3] = {vx[i], vy[i], vz[i]};
        double x0 = x[i], y0 = y[i], z0 = z[i];
        if (p->flags & OR_F_PUSH) {
            if (q[i] > 0) {
                double B[3], Ef[3];
                or_bfield(p, x0, y0, z0, B);
                or_efield(p, E, x0, y0, z0, Ef);
                or_boris(q[i] * OR_QE / M, Ef, B, dt, v);
            }
        }
        double x1 = x0, y1 = y0, z1 = z0;
        if (p->flags & OR_F_PUSH) { x1 = x0 + v[0] * dt; y1 = y0 + v[1] * dt; z1 = z0 + v[2] * dt; }
        vx[i] = v[0]; vy[i] = v[1]; vz[i] = v[2];
        x[i] = x1; y[i] = y1; z[i] = z1;

        /* 2. boundary test: first crossing along the straight segment */
        double r1 = sqrt(x1 * x1 + y1 * y1);
        if (fabs(r1 - p->R0) < gband || fabs(z1) < gband || fabs(z1 - p->L) < gband)
            guard[i] |= OR_G_BOUNDARY;
        int out_r = x1 * x1 + y1 * y1 > p->R0 * p->R0;
        int out_0 = z1 < 0.0, out_L = z1 > p->L;
        if (out_r || out_0 || out_L) {
            double fbest = 2.0, fr = 3.0, fz = 3.0;
            int kind = OR_LEAVE_NONE;
            double dx = x1 - x0, dy = y1 - y0, dz = z1 - z0;
            if (out_r) {
                double a = dx * dx + dy * dy, b = x0 * dx + y0 * dy, c = x0 * x0 + y0 * y0 - p->R0 * p->R0;
                double disc = sqrt(fmax(0.0, b * b - a * c));
                double f = (b + disc > 0.0) ? -c / (b + disc) : 0.0;
                if (f < 0.0) f = 0.0;
                fr = f;
                if (f < fbest) { fbest = f; kind = OR_LEAVE_RADIAL; }
            }
            if (out_0) {
                double f = z0 / (z0 - z1);
                fz = f;
                if (f < fbest) { fbest = f; kind = OR_LEAVE_Z0; }
            }
            if (out_L) {
                double f = (p->L - z0) / (z1 - z0);
                fz = f;
                if (f < fbest) { fbest = f; kind = OR_LEAVE_ZL; }
            }
            /* a step through a corner: which wall comes first is a rounding tie */
            if (fabs(fr - fz) < 1e-4) guard[i] |= OR_G_BOUNDARY;
            double cx = x0 + fbest * dx, cy = y0 + fbest * dy, cz = z0 + fbest * dz;
            if (kind == OR_LEAVE_ZL) {
                double rc = sqrt(cx * cx + cy * cy);
                if (fabs(rc - p->r_ap) < gband) guard[i] |= OR_G_BOUNDARY;
                if (rc * rc < p->r_ap * p->r_ap) kind = OR_LEAVE_APERTURE;
            }
            leave[i] = (uint8_t)kind;
            xc[3 * i] = cx; xc[3 * i + 1] = cy; xc[3 * i + 2] = cz;
            continue;
        }

        /* 3. MCC in the particle's cell */
        uint32_t g = 0;
        int64_t c = or_cell(p, x1, y1, z1, &g);
        guard[i] |= (uint8_t)g;
        cell[i] = c;
        uint32_t w[4];
        or_words(p->seed, (uint32_t)i, step, 0, w);
        double ne_c = ne[c];
        int zc = zone[c];
        int Q = q[i];
        /* step-wise ionisation Q -> Q+1, probability 1 - exp(-n_e k_Q(T_e) dt);
         * with double ionisation, Q -> Q+1 or Q+2 (or_ion_outcome) */
        if (((p->flags & OR_F_IONIZE) && Q < p->qmax) || ((p->flags & OR_F_RECOMB) && Q >= 1)) {
            int near = 0;
            int up = or_ion_outcome(p, ne_c, zc, rates, rates2, ratesr, Q, w[0], &near);
            if (near) guard[i] |= OR_G_IONIZE;
            if (up > 0) { Q += up; events[i] |= OR_EV_IONIZE; }
            if (up < 0) { Q -= 1; events[i] |= OR_EV_RECOMB; }
        }
        /* charge exchange with the neutral background: sigma_Q = Q sigma_1,
         * rate n0 sigma_Q v_rel, v_rel^2 = |v|^2 + 8 kT0/(pi M); Q = 2 is
         * forbidden; Q = 1 (resonant) gives a thermal ion; Q >= 3 -> Q-1 with
         * half of the release energy as an isotropic kick */
        /* with elastic scattering, charge exchange and elastic scattering
         * compete: one step's probability of either is 1 - exp(-n0 (sigma_cx +
         * sigma_el) v_rel dt), shared in proportion to the cross sections; the
         * word w1 below the charge-exchange threshold exchanges, between the
         * two thresholds it scatters elastically */
        int elastic = 0;
        if ((p->flags & OR_F_ELASTIC) && p->n0_m3 > 0.0 && Q >= 1 && p->sigma_el_m2 > 0.0) {
            double scx = ((p->flags & OR_F_CX) && Q != 2) ? p->sigma1_m2 * Q : 0.0;
            double sel = p->sigma_el_m2 * Q;
            double vrel = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2] + 8.0 * p->T0_eV * OR_QE / (OR_PI * M));
            double pt = -expm1(-p->n0_m3 * (scx + sel) * vrel * dt);
            double thr = or_threshold(pt), thr1 = or_threshold(pt * (scx / (scx + sel)));
            if (fabs((double)w[1] - thr) < 1e-5 * thr + 2.0 || fabs((double)w[1] - thr1) < 1e-5 * thr1 + 2.0)
                guard[i] |= OR_G_CX;
            if ((double)w[1] >= floor(thr1) && (double)w[1] < floor(thr)) elastic = 1;
        }
        if (elastic) {
            /* isotropic in the centre-of-mass frame with a background atom
             * drawn from the Maxwellian at T0 (stream-3 words); the new
             * direction of the relative velocity from the stream-2 words (the
             * wall stream, unused by a particle that stayed inside) */
            uint32_t u[4], d[4];
            or_words(p->seed, (uint32_t)i, step, 3, u);
            or_words(p->seed, (uint32_t)i, step, 2, d);
            double r1g = sig0 * sqrt(-2.0 * log(or_unit(u[0])));
            double t1 = 2.0 * OR_PI * or_unit(u[1]);
            double r2g = sig0 * sqrt(-2.0 * log(or_unit(u[2])));
            double t2 = 2.0 * OR_PI * or_unit(u[3]);
            double va[3] = {r1g * cos(t1), r1g * sin(t1), r2g * cos(t2)};
            double gx = v[0] - va[0], gy = v[1] - va[1], gz = v[2] - va[2];
            double gm = sqrt(gx * gx + gy * gy + gz * gz);
            double ct = 2.0 * or_unit(d[0]) - 1.0;
            double st = sqrt(fmax(0.0, 1.0 - ct * ct));
            double ph = 2.0 * OR_PI * or_unit(d[1]);
            double n[3] = {st * cos(ph), st * sin(ph), ct};
            for (int k = 0; k < 3; ++k) v[k] = 0.5 * (v[k] + va[k]) + 0.5 * gm * n[k];
            events[i] |= OR_EV_ELASTIC;
        } else if ((p->flags & OR_F_CX) && p->n0_m3 > 0.0 && Q >= 1 && Q != 2) {
            double vrel = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2] + 8.0 * p->T0_eV * OR_QE / (OR_PI * M));
            double pr = -expm1(-p->n0_m3 * p->sigma1_m2 * Q * vrel * dt);
            if ((p->flags & OR_F_ELASTIC) && p->sigma_el_m2 > 0.0) {
                /* the exchange threshold of the shared word, as above */
                double sel = p->sigma_el_m2 * Q, scx = p->sigma1_m2 * Q;
                pr = -expm1(-p->n0_m3 * (scx + sel) * vrel * dt) * (scx / (scx + sel));
            }
            double thr = or_threshold(pr);
            if (fabs((double)w[1] - thr) < 1e-5 * thr + 2.0) guard[i] |= OR_G_CX;
            if ((double)w[1] < floor(thr)) {
                uint32_t u[4];
                or_words(p->seed, (uint32_t)i, step, 3, u);
                events[i] |= OR_EV_CX;
                if (Q == 1) {
                    double r1g = sig0 * sqrt(-2.0 * log(or_unit(u[0])));
                    double t1 = 2.0 * OR_PI * or_unit(u[1]);
                    double r2g = sig0 * sqrt(-2.0 * log(or_unit(u[2])));
                    double t2 = 2.0 * OR_PI * or_unit(u[3]);
                    v[0] = r1g * cos(t1); v[1] = r1g * sin(t1); v[2] = r2g * cos(t2);
                } else {
                    double dv = sqrt(2.0 * 0.5 * p->E_cx_eV * OR_QE / M);
                    double ct = 2.0 * or_unit(u[0]) - 1.0;
                    double st = sqrt(fmax(0.0, 1.0 - ct * ct));
                    double ph = 2.0 * OR_PI * or_unit(u[1]);
                    v[0] += dv * st * cos(ph); v[1] += dv * st * sin(ph); v[2] += dv * ct;
                    Q -= 1;
                }
            }
        }
        /* electron-ion heating kick: |dV| = D, direction (R + delta)/|R + delta|
         * with R an isotropic unit vector; D^2 = 3.715e-6 n_e lnL_ei Q^p dt /
         * (M^2 sqrt(T_e)), SI with M in amu and T_e in eV */
        if ((p->flags & OR_F_EIKICK) && Q >= 1) {
            double Te = zc ? p->Te_warm : p->Te_cold;
            double qp = p->ei_charge_power == 1 ? (double)Q : (double)Q * Q;
            double D = sqrt(3.715e-6 * ne_c * p->lnL_ei * qp * dt /
                            (p->mass_amu * p->mass_amu * sqrt(Te)));
            double ct = 2.0 * or_unit(w[2]) - 1.0;
            double st = sqrt(fmax(0.0, 1.0 - ct * ct));
            double ph = 2.0 * OR_PI * or_unit(w[3]);
            double R[3] = {st * cos(ph), st * sin(ph), ct};
            double d[3] = {R[0] + dlx[c], R[1] + dly[c], R[2]};
            double dm = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            if (dm > 0.0)
                for (int k = 0; k < 3; ++k) v[k] += D * d[k] / dm;
        }
        if ((guard[i] & OR_G_CELL) &&
            or_cell_record_guard(p, x1, y1, z1, c, ne, zone, dlx, dly, rates, rates2, ratesr, q[i], Q, w[0]))
            guard[i] |= OR_G_CELLREC;
        q[i] = Q;
        vx[i] = v[0]; vy[i] = v[1]; vz[i] = v[2];
        if (Q >= 1) part[i] = 1;
    }

    /* phase 2: ion-ion Coulomb collisions among the ions that stayed */
    if (p->flags & OR_F_COULOMB) or_coulomb(p, n, cell, part, vx, vy, vz, q, step, dt, events, t);

    /* phase 3: wall / aperture bookkeeping of the particles that left (in
     * particle order: the FP64 energy tally adds in a fixed order) */
    for (int64_t i = 0; i < n; ++i) {
        if (status[i] & 1u) continue;
        if (leave[i] != OR_LEAVE_NONE) {
            int Q = q[i];
            qleave[i] = Q;
            if (Q >= 1)
                t->ke_lost_eV += 0.5 * M * (vx[i] * vx[i] + vy[i] * vy[i] + vz[i] * vz[i]) / OR_QE;
            double cx = xc[3 * i], cy = xc[3 * i + 1], cz = xc[3 * i + 2];
            double nrm[3], e1[3], e2[3];
            if (leave[i] == OR_LEAVE_APERTURE) {
                t->extracted[Q] += 1;
                t->r_ext_sum[Q] += sqrt(cx * cx + cy * cy);
                events[i] |= OR_EV_EXTRACT;
                cx = p->inlet[0]; cy = p->inlet[1]; cz = p->inlet[2];
                nrm[0] = 0; nrm[1] = 0; nrm[2] = 1; e1[0] = 1; e1[1] = 0; e1[2] = 0; e2[0] = 0; e2[1] = 1; e2[2] = 0;
            } else {
                t->lost[Q] += 1;
                events[i] |= OR_EV_WALL;
                if (leave[i] == OR_LEAVE_RADIAL) {
                    double rc = sqrt(cx * cx + cy * cy);
                    double sc = (p->R0 - eps_wall) / rc;
                    double ux = cx / rc, uy = cy / rc;
                    cx *= sc; cy *= sc;
                    nrm[0] = -ux; nrm[1] = -uy; nrm[2] = 0;
                    e1[0] = -uy; e1[1] = ux; e1[2] = 0;
                    e2[0] = 0; e2[1] = 0; e2[2] = 1;
                } else if (leave[i] == OR_LEAVE_Z0) {
                    cz = eps_wall;
                    nrm[0] = 0; nrm[1] = 0; nrm[2] = 1; e1[0] = 1; e1[1] = 0; e1[2] = 0; e2[0] = 0; e2[1] = 1; e2[2] = 0;
                } else {
                    cz = p->L - eps_wall;
                    nrm[0] = 0; nrm[1] = 0; nrm[2] = -1; e1[0] = 1; e1[1] = 0; e1[2] = 0; e2[0] = 0; e2[1] = 1; e2[2] = 0;
                }
            }
            q[i] = 0;
            if (p->flags & OR_F_RECYCLE) {
                uint32_t w[4];
                double v[3];
                or_words(p->seed, (uint32_t)i, step, 2, w);
                or_emit(Q >= 1 && leave[i] != OR_LEAVE_APERTURE ? sig_refl : sig0, nrm, e1, e2, w, v);
                x[i] = cx; y[i] = cy; z[i] = cz;
                vx[i] = v[0]; vy[i] = v[1]; vz[i] = v[2];
            } else {
                status[i] |= 1u;
                continue;
            }
        }
    }
    /* phase 4: NGP deposition at the final positions (integer sums, so the
     * order of the additions does not matter) */
    if (dep_count) {
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            if (status[i] & 1u) continue;
            int64_t c = or_cell(p, x[i], y[i], z[i], NULL);
#pragma omp atomic
            dep_count[c] += 1;
#pragma omp atomic
            dep_charge[c] += q[i];
        }
    }
    free(cell); free(leave); free(part); free(xc); free(qleave);
}
