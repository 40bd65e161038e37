"""Seeded synthetic inputs for the ECRIS ion time step.

This module only builds input data: species tables, run parameters, initial
particle states, per-cell electron-density draws and a synthetic electric-field
grid.  It holds none of the method's arithmetic (no field evaluation, no push,
no rates, no collisions), so the FP64 oracle and the CUDA path can both take
their inputs from it without sharing any of the computation.

The paper (Sec. II) models argon in five real sources whose Poisson-Superfish
field maps, ionisation-rate datasets [20-23] and charge-exchange cross sections
[17,18] are not available.  Every table here is therefore a documented
synthetic stand-in with the shapes and magnitudes of the paper's workloads:

* species: mass, highest charge state, and an ionisation-potential ladder from a
  screened-hydrogenic rule (synthetic, not measured data);
* geometry and mirror/hexapole field extremes as in the paper's Table I;
* 2e5-class particle ensembles with ~75 % atoms (Sec. II), Maxwellian
  velocities at the gas temperature.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

# Physical constants used only to draw thermal velocities of the inputs.
E_CHARGE = 1.602176634e-19
AMU = 1.66053906660e-27
RYDBERG_EV = 13.605693122994

# Process switches (mirrors the C header's ECRIS_F_* values).
F_PUSH = 1 << 0
F_IONIZE = 1 << 1
F_CX = 1 << 2
F_EIKICK = 1 << 3
F_COULOMB = 1 << 4
F_RECYCLE = 1 << 5
F_ISOHEAT = 1 << 6   # heating kick without the drift bias (delta = 0)
F_DOUBLE = 1 << 7    # double ionisation Q -> Q+2
F_ELASTIC = 1 << 8   # elastic ion-atom scattering
F_RECOMB = 1 << 9    # radiative recombination Q -> Q-1
F_ALL_NO_COULOMB = F_PUSH | F_IONIZE | F_CX | F_EIKICK | F_RECYCLE
F_ALL = F_ALL_NO_COULOMB | F_COULOMB


@dataclasses.dataclass(frozen=True)
class Species:
    """A synthetic ion species: mass, nuclear charge and ionisation ladder."""

    name: str
    mass_amu: float
    Z: int
    qmax: int

    def ladder(self):
        """Ionisation potentials P_Q (eV) and outer-shell counts q_Q, Q=0..qmax-1.

        Synthetic rule: the electron removed from an ion with Z-Q electrons
        sits in the outermost occupied shell n (shells filled in order with
        capacity 2n^2); it sees z_eff = Z - N_inner - (N_same - 1)/2, where
        N_inner counts electrons in lower shells and N_same those in shell n,
        and P_Q = Ry z_eff^2 / n^2.  q_Q = N_same is the number of equivalent
        outer electrons.  For Ar this gives 31, 38, ... 4.4e3 eV, close in
        magnitude to the real ladder but not measured data.
        """
        ip = np.zeros(self.qmax, dtype=np.float64)
        nout = np.zeros(self.qmax, dtype=np.int32)
        for q in range(self.qmax):
            ne = self.Z - q
            shells = []
            left = ne
            n = 1
            while left > 0:
                take = min(left, 2 * n * n)
                shells.append(take)
                left -= take
                n += 1
            n_out = len(shells)
            n_same = shells[-1]
            n_inner = ne - n_same
            zeff = self.Z - n_inner - 0.5 * (n_same - 1)
            ip[q] = RYDBERG_EV * zeff * zeff / (n_out * n_out)
            nout[q] = n_same
        return ip, nout


ARGON = Species("Ar", 40.0, 18, 18)
OXYGEN = Species("O", 16.0, 8, 8)
KRYPTON = Species("Kr", 84.0, 36, 36)
SPECIES = {"Ar": ARGON, "O": OXYGEN, "Kr": KRYPTON}


@dataclasses.dataclass
class RunParams:
    """All scalar inputs of one run (SI units unless the name says otherwise)."""

    species: Species = ARGON
    # geometry (Table I shapes): cylinder radius and length, aperture radius
    R0: float = 0.032
    L: float = 0.30
    r_ap: float = 0.005
    inlet: tuple = (0.016, 0.0, 3.0e-7)
    # on-axis mirror extremes and hexapole at the wall (T); ECR field 0.5 T at 14 GHz
    B_inj: float = 2.2
    B_min: float = 0.4
    B_ext: float = 1.1
    B_hex: float = 1.0
    B_ecr: float = 0.5
    # mesh
    nx: int = 32
    ny: int = 32
    nz: int = 64
    # electrons: density inside / outside the ECR zone (cm^-3), temperatures (eV)
    ne_in_cm3: float = 1e11
    ne_out_cm3: float = 5e9
    Te_warm_eV: float = 1000.0
    Te_cold_eV: float = 5.0
    # neutrals and collisions
    n0_cm3: float = 0.0
    T0_eV: float = 0.026
    sigma1_cm2: float = 3e-15
    E_cx_eV: float = 10.0
    lnL_ii: float = 10.0
    lnL_ei: float = 17.0
    ei_charge_power: int = 2
    # optional on-axis field table: B0 (T) at z_k = k L/(n-1), n >= 4; None:
    # the synthetic mirror through B_inj, B_min, B_ext
    B_axial: Optional[tuple] = None
    # opt-in processes: re-emission temperature of ions neutralised at a wall
    # (0: T0), synthetic elastic ion-atom cross section of Q = 1 (cm^2),
    # double- and triple-ionisation rate factors (k3_factor = 0: no triple)
    T_refl_eV: float = 0.0
    sigma_el1_cm2: float = 4e-15
    k2_factor: float = 0.1
    k3_factor: float = 0.0
    flags: int = F_ALL_NO_COULOMB
    # macroparticle weight and RNG key
    weight: float = 1e8
    seed: int = 1
    dt: float = 1e-9

    @property
    def ncells(self) -> int:
        return self.nx * self.ny * self.nz


@dataclasses.dataclass
class Workload:
    """A named synthetic workload: run parameters plus the ensemble recipe."""

    name: str
    params: RunParams
    n: int
    steps: int
    atom_fraction: float = 1.0     # fraction of particles starting as atoms
    ion_qmax_init: int = 0         # initial ions drawn uniformly in 1..ion_qmax_init
    ion_T_eV: float = 0.25         # initial ion temperature
    zone_box: tuple = (0.018, 0.157, 0.213)  # (r, z_lo, z_hi) that ions/atoms start in
    atoms_fill_chamber: bool = False
    ne_cells_loguniform: Optional[tuple] = None  # (lo, hi) cm^-3 per cell inside the zone
    efield: Optional[tuple] = None  # (a, b): E = (a x, a y, b (z - L/2)) V/m


def config_small(seed: int = 1, n: int = 10_000, steps: int = 1000) -> Workload:
    """Single plain run: Ar, 1e4 atoms in the ECR zone, 32x32x64 grid, 1e3 steps."""
    p = RunParams(seed=seed, n0_cm3=0.0, flags=F_ALL_NO_COULOMB)
    return Workload("ar_1e4_32x32x64", p, n=n, steps=steps)


def config_scaled(seed: int = 2, n: int = 4_000_000, steps: int = 10_000) -> Workload:
    """Scaled plain run: Ar, 4e6 particles, 64x64x128 grid, n0=1e10, Coulomb on.

    Ensemble recipe: 75 % atoms filling the chamber (Sec. II), 25 % ions with Q
    uniform in 1..12 inside the zone box; ne per zone cell log-uniform in
    1e11-1e12 cm^-3.
    """
    p = RunParams(seed=seed, nx=64, ny=64, nz=128, n0_cm3=1e10, flags=F_ALL)
    return Workload("ar_4e6_64x64x128_coulomb", p, n=n, steps=steps,
                    atom_fraction=0.75, ion_qmax_init=12, atoms_fill_chamber=True,
                    ne_cells_loguniform=(1e11, 1e12))


def config_oxygen_scan(i: int, n: Optional[int] = None) -> Workload:
    """One run of the batched gas-flow scan: O (Q=0..8), n0 swept 3e9-3e11 cm^-3."""
    rng = np.random.default_rng(1000 + i)
    if n is None:
        n = int(round(math.exp(rng.uniform(math.log(2e5), math.log(2e6)))))
    n0 = 3e9 * (3e11 / 3e9) ** (i / 63.0)
    p = RunParams(species=OXYGEN, seed=1000 + i, n0_cm3=n0, flags=F_ALL_NO_COULOMB)
    return Workload(f"o_scan_{i}", p, n=n, steps=10_000, atom_fraction=0.75,
                    ion_qmax_init=6, atoms_fill_chamber=True)


def config_power_scan(i: int, n: Optional[int] = None) -> Workload:
    """One run of the batched microwave-power scan: Ar, electron density in the
    zone log-uniform 5e10-2e12 cm^-3 and warm-electron temperature log-uniform
    0.3-3 keV (the coupled power sets both, Sec. II), N log-uniform 1e5-4e6."""
    rng = np.random.default_rng(2000 + i)
    lu = lambda lo, hi: math.exp(rng.uniform(math.log(lo), math.log(hi)))
    ne, te = lu(5e10, 2e12), lu(300.0, 3000.0)
    n_draw = int(round(lu(1e5, 4e6)))
    p = RunParams(seed=2000 + i, ne_in_cm3=ne, Te_warm_eV=te, n0_cm3=1e10, flags=F_ALL)
    return Workload(f"ar_power_scan_{i}", p, n=n_draw if n is None else n, steps=10_000,
                    atom_fraction=0.75, ion_qmax_init=8, atoms_fill_chamber=True)


SERVED_MESHES = ((32, 32, 64), (64, 64, 128), (96, 96, 192))


def served_stream(seed: int = 5, rate_per_s: float = 20.0, duration_s: float = 2.0,
                  n_range: tuple = (1e4, 8e6), dt: float = 1e-7):
    """A served request stream: Poisson arrivals (rate_per_s) over duration_s.

    Each request is a parameter-scan run: species uniform over O, Ar, Kr;
    N log-uniform in n_range; mesh uniform over SERVED_MESHES; neutral density
    (gas flow) log-uniform 3e9-3e11 cm^-3; zone electron density log-uniform
    5e10-2e12 cm^-3 and warm-electron temperature 0.3-3 keV (microwave power);
    every process of the step on; time step dt (0.1 us by default: 4096 steps
    span 0.4 ms, about one ion confinement time, and a 256-step window of a
    run of a few 1e5 particles or more extracts the 400 ions the convergence
    rule asks for).  Returns a list of (arrival time s, Workload).
    """
    rng = np.random.default_rng(seed)
    lu = lambda lo, hi: math.exp(rng.uniform(math.log(lo), math.log(hi)))
    out, t, i = [], 0.0, 0
    species = (OXYGEN, ARGON, KRYPTON)
    while True:
        t += rng.exponential(1.0 / rate_per_s)
        if t > duration_s:
            return out
        sp = species[int(rng.integers(3))]
        nx, ny, nz = SERVED_MESHES[int(rng.integers(len(SERVED_MESHES)))]
        n = int(round(lu(*n_range)))
        p = RunParams(species=sp, nx=nx, ny=ny, nz=nz, n0_cm3=lu(3e9, 3e11), ne_in_cm3=lu(5e10, 2e12),
                      Te_warm_eV=lu(300.0, 3000.0), flags=F_ALL, seed=5000 + i, dt=dt)
        out.append((t, Workload(f"served_{i}_{sp.name}", p, n=n, steps=4096, atom_fraction=0.75,
                                ion_qmax_init=min(8, sp.qmax - 1), atoms_fill_chamber=True)))
        i += 1


def _mb_velocities(rng, n, T_eV, mass_amu):
    sigma = math.sqrt(T_eV * E_CHARGE / (mass_amu * AMU))
    return rng.normal(0.0, sigma, size=(3, n))


def flat_axial_profile(rp: RunParams, n: int = 513, flat: float = 0.06):
    """Samples of a synthetic flat on-axis profile (the paper's flat
    configuration, Sec. IV, Fig. 34): the mirror's two raised-cosine halves
    moved apart by a plateau of length `flat` at B_min, centred where the
    plain mirror has its minimum.  B0 at z_k = k L/(n-1) as a tuple."""
    zm = rp.L / (1.0 + np.sqrt((rp.B_ext - rp.B_min) / (rp.B_inj - rp.B_min)))
    z1, z2 = zm - 0.5 * flat, zm + 0.5 * flat
    z = np.linspace(0.0, rp.L, n)
    b = np.full(n, rp.B_min)
    lo, hi = z < z1, z > z2
    b[lo] = rp.B_min + 0.5 * (rp.B_inj - rp.B_min) * (1.0 + np.cos(np.pi * z[lo] / z1))
    b[hi] = rp.B_min + 0.5 * (rp.B_ext - rp.B_min) * (1.0 - np.cos(np.pi * (z[hi] - z2) / (rp.L - z2)))
    return tuple(float(v) for v in b)


def make_particles(wl: Workload, seed: Optional[int] = None):
    """Initial state of a workload: dict of float32 x,y,z,vx,vy,vz and uint8 q.

    Particles start uniformly inside the zone box (a cylinder r < r_z,
    z_lo < z < z_hi standing in for the ECR surface) or, for atoms when
    `atoms_fill_chamber`, uniformly in the whole chamber.  Velocities are
    Maxwellian: atoms at T0, ions at `ion_T_eV`.
    """
    p = wl.params
    rng = np.random.default_rng(p.seed if seed is None else seed)
    n = wl.n
    is_ion = rng.random(n) >= wl.atom_fraction
    q = np.zeros(n, dtype=np.uint8)
    if wl.ion_qmax_init > 0:
        q[is_ion] = rng.integers(1, wl.ion_qmax_init + 1, size=int(is_ion.sum()))
    r_z, z_lo, z_hi = wl.zone_box
    rad = np.where(is_ion | (not wl.atoms_fill_chamber), r_z, p.R0 * (1 - 1e-3))
    zlo = np.where(is_ion | (not wl.atoms_fill_chamber), z_lo, p.L * 1e-3)
    zhi = np.where(is_ion | (not wl.atoms_fill_chamber), z_hi, p.L * (1 - 1e-3))
    rr = rad * np.sqrt(rng.random(n))
    th = rng.random(n) * 2 * math.pi
    x = rr * np.cos(th)
    y = rr * np.sin(th)
    z = zlo + (zhi - zlo) * rng.random(n)
    v_atom = _mb_velocities(rng, n, p.T0_eV, p.species.mass_amu)
    v_ion = _mb_velocities(rng, n, wl.ion_T_eV, p.species.mass_amu)
    v = np.where(is_ion[None, :], v_ion, v_atom)
    f32 = np.float32
    return {
        "x": x.astype(f32), "y": y.astype(f32), "z": z.astype(f32),
        "vx": v[0].astype(f32), "vy": v[1].astype(f32), "vz": v[2].astype(f32),
        "q": q,
    }


def make_ne_cells(wl: Workload, seed: Optional[int] = None):
    """Per-cell electron density (cm^-3) used inside the ECR zone, or None.

    Drawn i.i.d. log-uniform per cell from `ne_cells_loguniform`; cells outside
    the zone ignore it.  Layout: x fastest, then y, then z (Nc float32).
    """
    if wl.ne_cells_loguniform is None:
        return None
    lo, hi = wl.ne_cells_loguniform
    rng = np.random.default_rng((wl.params.seed if seed is None else seed) + 7919)
    u = rng.random(wl.params.ncells)
    return np.exp(math.log(lo) + (math.log(hi) - math.log(lo)) * u).astype(np.float32)


def make_efield(p: RunParams, a: float, b: float):
    """Cell-centred synthetic E grid, E = (a x, a y, b (z - L/2)) V/m, shape (Nc, 3).

    The field is linear in position, so trilinear interpolation between cell
    centres reproduces it exactly away from the outer half cells.  Layout: x
    fastest, then y, then z.
    """
    dx = 2 * p.R0 / p.nx
    dy = 2 * p.R0 / p.ny
    dz = p.L / p.nz
    xc = -p.R0 + (np.arange(p.nx) + 0.5) * dx
    yc = -p.R0 + (np.arange(p.ny) + 0.5) * dy
    zc = (np.arange(p.nz) + 0.5) * dz
    Z, Y, X = np.meshgrid(zc, yc, xc, indexing="ij")
    E = np.stack([a * X, a * Y, b * (Z - p.L / 2)], axis=-1)
    return E.reshape(-1, 3).astype(np.float32)
