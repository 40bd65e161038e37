"""Python access to the FP64 CPU oracle (test infrastructure only).

Only the tests, the smoke check and the benchmark's timed CPU-baseline leg may
import this module.  It compiles `ecris_oracle.c` with gcc into a shared
library beside it and wraps it with ctypes.  The oracle shares no code with the
CUDA path: its inputs come from `paper_1507_03392_gb300.inputs` and nothing
else.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ecris_oracle.c")
LIB = os.path.join(HERE, "libecris_oracle.so")

F_PUSH, F_IONIZE, F_CX, F_EIKICK, F_COULOMB, F_RECYCLE = 1, 2, 4, 8, 16, 32
F_ISOHEAT, F_DOUBLE, F_ELASTIC, F_RECOMB = 64, 128, 256, 512
EV_WALL, EV_EXTRACT, EV_IONIZE, EV_CX, EV_COULOMB, EV_ELASTIC, EV_RECOMB = 1, 2, 4, 8, 16, 32, 64
G_CELL, G_BOUNDARY, G_IONIZE, G_CX, G_CELLREC = 1, 2, 4, 8, 16
# guards that can change a single-particle outcome (no Coulomb pairing)
G_SINGLE = G_BOUNDARY | G_IONIZE | G_CX | G_CELLREC
QMAX_SLOTS = 64
FPTD_BINS = 120


def fptd_bin(age: int) -> int:
    """Log bin of a first-passage age in steps (>= 1): e = floor(log2 age),
    m = the two bits below the leading one, bin = 4 e + m."""
    e = int(age).bit_length() - 1
    m = (age >> (e - 2)) & 3 if e >= 2 else (age << (2 - e)) & 3
    return 4 * e + m


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, FP64, OpenMP over particles)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
               "-ffp-contract=off", SRC, "-o", LIB, "-lm"]
        subprocess.run(cmd, check=True)
    return LIB


class Params(ctypes.Structure):
    _fields_ = [
        ("R0", ctypes.c_double), ("L", ctypes.c_double), ("r_ap", ctypes.c_double),
        ("inlet", ctypes.c_double * 3),
        ("B_inj", ctypes.c_double), ("B_min", ctypes.c_double), ("B_ext", ctypes.c_double),
        ("B_hex", ctypes.c_double), ("B_ecr", ctypes.c_double),
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("qmax", ctypes.c_int32),
        ("mass_amu", ctypes.c_double),
        ("Te_warm", ctypes.c_double), ("Te_cold", ctypes.c_double),
        ("n0_m3", ctypes.c_double), ("T0_eV", ctypes.c_double), ("sigma1_m2", ctypes.c_double),
        ("E_cx_eV", ctypes.c_double), ("lnL_ii", ctypes.c_double), ("lnL_ei", ctypes.c_double),
        ("ei_charge_power", ctypes.c_int32), ("flags", ctypes.c_uint32),
        ("weight", ctypes.c_double), ("seed", ctypes.c_uint64), ("dt", ctypes.c_double),
        ("T_refl_eV", ctypes.c_double), ("sigma_el_m2", ctypes.c_double), ("k2_factor", ctypes.c_double),
        ("k3_factor", ctypes.c_double),
        ("ax_n", ctypes.c_int32), ("ax_y", ctypes.c_void_p), ("ax_M", ctypes.c_void_p),
    ]


class Tally(ctypes.Structure):
    _fields_ = [
        ("extracted", ctypes.c_int64 * QMAX_SLOTS),
        ("lost", ctypes.c_int64 * QMAX_SLOTS),
        ("ke_lost_eV", ctypes.c_double),
        ("coulomb_pairs", ctypes.c_int64),
        ("r_ext_sum", ctypes.c_double * QMAX_SLOTS),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        d, i32, u32, i64, p = (ctypes.c_double, ctypes.c_int32, ctypes.c_uint32,
                               ctypes.c_int64, ctypes.c_void_p)
        pp = ctypes.POINTER(Params)
        _lib.or_philox.argtypes = [p, p, p]
        _lib.or_zmin.argtypes = [pp]
        _lib.or_zmin.restype = d
        _lib.or_b0.argtypes = [pp, d, p]
        _lib.or_bfield.argtypes = [pp, d, d, d, p]
        _lib.or_efield.argtypes = [pp, p, d, d, d, p]
        _lib.or_lotz_rate.argtypes = [d, ctypes.c_int, d]
        _lib.or_lotz_rate.restype = d
        _lib.or_build_rates.argtypes = [pp, p, p, p]
        _lib.or_build_rates2.argtypes = [pp, p, p, p]
        _lib.or_axial_setup.argtypes = [ctypes.c_int32, d, p, p]
        _lib.or_build_rates_rec.argtypes = [pp, p]
        _lib.or_set_threads.argtypes = [ctypes.c_int]
        _lib.or_set_threads.restype = ctypes.c_int
        _lib.or_recomb_rate.argtypes = [ctypes.c_int, d]
        _lib.or_recomb_rate.restype = d
        _lib.or_setup_cells.argtypes = [pp, p, d, d, p, p, p, p, p]
        _lib.or_cell_delta.argtypes = [pp, p, p, p, p, p]
        _lib.or_boris.argtypes = [d, p, p, d, p]
        _lib.or_emit.argtypes = [d, p, p, p, p, p]
        _lib.or_nanbu_A.argtypes = [d]
        _lib.or_nanbu_A.restype = d
        _lib.or_nanbu_cos.argtypes = [d, d]
        _lib.or_nanbu_cos.restype = d
        _lib.or_nanbu_s.argtypes = [d, d, d, d, d, d, d]
        _lib.or_nanbu_s.restype = d
        _lib.or_scatter_pair.argtypes = [p, p, d, d]
        _lib.or_step.argtypes = [pp, p, p, p, p, p, p, p, p, i64, p, p, p, p, p, p, p, p, u32, p, p,
                                 ctypes.POINTER(Tally), p, p]
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def philox(ctr, key):
    """Philox4x32-10 of a 4-word counter and 2-word key -> 4 uint32 words."""
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().or_philox(_ptr(c), _ptr(k), _ptr(out))
    return out


def make_params(rp, dt=None) -> Params:
    """Oracle parameter block from an `inputs.RunParams` (cm units converted to SI)."""
    p = Params()
    p.R0, p.L, p.r_ap = rp.R0, rp.L, rp.r_ap
    for k in range(3):
        p.inlet[k] = rp.inlet[k]
    p.B_inj, p.B_min, p.B_ext, p.B_hex, p.B_ecr = rp.B_inj, rp.B_min, rp.B_ext, rp.B_hex, rp.B_ecr
    p.nx, p.ny, p.nz, p.qmax = rp.nx, rp.ny, rp.nz, rp.species.qmax
    p.mass_amu = rp.species.mass_amu
    p.Te_warm, p.Te_cold = rp.Te_warm_eV, rp.Te_cold_eV
    p.n0_m3 = rp.n0_cm3 * 1e6
    p.T0_eV = rp.T0_eV
    p.sigma1_m2 = rp.sigma1_cm2 * 1e-4
    p.E_cx_eV, p.lnL_ii, p.lnL_ei = rp.E_cx_eV, rp.lnL_ii, rp.lnL_ei
    p.ei_charge_power = rp.ei_charge_power
    p.flags = rp.flags
    p.weight = rp.weight
    p.seed = rp.seed
    p.dt = rp.dt if dt is None else dt
    p.T_refl_eV = rp.T_refl_eV
    p.sigma_el_m2 = rp.sigma_el1_cm2 * 1e-4
    p.k2_factor = rp.k2_factor
    p.k3_factor = rp.k3_factor
    if rp.B_axial is not None:
        # on-axis table: the spline's second derivatives, kept alive with p
        y = np.ascontiguousarray(rp.B_axial, dtype=np.float64)
        M = np.zeros_like(y)
        lib().or_axial_setup(len(y), rp.L, _ptr(y), _ptr(M))
        p.ax_n, p.ax_y, p.ax_M = len(y), y.ctypes.data, M.ctypes.data
        p._keep = (y, M)
    return p


def bfield(p: Params, x, y, z):
    out = np.zeros(3)
    lib().or_bfield(ctypes.byref(p), float(x), float(y), float(z), _ptr(out))
    return out


def b0(p: Params, z):
    out = np.zeros(3)
    lib().or_b0(ctypes.byref(p), float(z), _ptr(out))
    return out


def lotz_rate(P_eV, q_outer, Te_eV):
    return lib().or_lotz_rate(float(P_eV), int(q_outer), float(Te_eV))


def boris(qm, E, B, dt, v):
    v = np.array(v, dtype=np.float64)
    lib().or_boris(float(qm), _ptr(np.asarray(E, np.float64)), _ptr(np.asarray(B, np.float64)),
                   float(dt), _ptr(v))
    return v


def ngp_cells(rp, x, y, z):
    """Nearest-grid-point cell of each position (ix fastest), by the floor of
    the coordinate over the mesh step; positions on the upper faces clamp."""
    dx, dy, dz = 2 * rp.R0 / rp.nx, 2 * rp.R0 / rp.ny, rp.L / rp.nz
    ix = np.clip(np.floor((np.asarray(x, np.float64) + rp.R0) / dx).astype(np.int64), 0, rp.nx - 1)
    iy = np.clip(np.floor((np.asarray(y, np.float64) + rp.R0) / dy).astype(np.int64), 0, rp.ny - 1)
    iz = np.clip(np.floor(np.asarray(z, np.float64) / dz).astype(np.int64), 0, rp.nz - 1)
    return (iz * rp.ny + iy) * rp.nx + ix


def probe_moments(rp, state, cells, alive=None):
    """Moments of the particles in each listed cell by charge state (Sec.
    III.A profiles): [len(cells), qmax + 1, 7] holding the count and the sums
    of vx, vy, vz, vx^2, vy^2, vz^2."""
    qs = rp.species.qmax + 1
    cells = np.asarray(cells, dtype=np.int64)
    out = np.zeros((len(cells), qs, 7))
    slot = np.full(rp.ncells, -1, dtype=np.int64)
    slot[cells] = np.arange(len(cells))
    s = slot[ngp_cells(rp, state["x"], state["y"], state["z"])]
    sel = s >= 0 if alive is None else (s >= 0) & alive
    q = np.asarray(state["q"], dtype=np.int64)
    v = [np.asarray(state[k], dtype=np.float64) for k in ("vx", "vy", "vz")]
    for i in np.nonzero(sel)[0]:
        row = out[s[i], q[i]]
        row[0] += 1.0
        for c in range(3):
            row[1 + c] += v[c][i]
            row[4 + c] += v[c][i] * v[c][i]
    return out


def moment_profiles(rp, moments, samples, weight=None):
    """Densities, temperatures and the ion pressure from summed moments
    (Sec. III.A): n_Q = w count / (samples V_cell) (m^-3), T_Q = M (<v^2> -
    <v>^2) / 3 in eV, P = sum over Q >= 1 of n_Q T_Q (eV m^-3) and the mean
    ion temperature P / sum over Q >= 1 of n_Q (eV).  Empty slots get T = 0."""
    w = rp.weight if weight is None else weight
    vol = (2.0 * rp.R0 / rp.nx) * (2.0 * rp.R0 / rp.ny) * (rp.L / rp.nz)
    cnt = moments[..., 0]
    n = w * cnt / (samples * vol)
    with np.errstate(invalid="ignore", divide="ignore"):
        mean_v2 = (moments[..., 4] + moments[..., 5] + moments[..., 6]) / cnt
        mean_v = moments[..., 1:4] / cnt[..., None]
        var = mean_v2 - (mean_v ** 2).sum(axis=-1)
        T = np.where(cnt > 0, rp.species.mass_amu * 1.66053906660e-27 * var / 3.0 / 1.602176634e-19, 0.0)
        P = (n[..., 1:] * T[..., 1:]).sum(axis=-1)
        ni = n[..., 1:].sum(axis=-1)
        Tm = np.where(ni > 0, P / ni, 0.0)
    return {"n": n, "T_eV": T, "P_eV_m3": P, "T_mean_eV": Tm}


def screen_hits(rp, state, slabs, pixels, alive=None):
    """Screen images (Sec. III.A, Figs. 9-11, 16): for each slab z_lo <= z <
    z_hi, one hit per particle in it on the pixel under it, by charge state,
    pixels x pixels over [-R0, R0)^2: [len(slabs), qmax + 1, py, px]."""
    qs = rp.species.qmax + 1
    out = np.zeros((len(slabs), qs, pixels, pixels), dtype=np.int64)
    x, y, z = (np.asarray(state[k], dtype=np.float64) for k in ("x", "y", "z"))
    q = np.asarray(state["q"], dtype=np.int64)
    px = np.floor((x + rp.R0) / (2 * rp.R0) * pixels).astype(np.int64)
    py = np.floor((y + rp.R0) / (2 * rp.R0) * pixels).astype(np.int64)
    for k, (lo, hi) in enumerate(slabs):
        sel = (z >= lo) & (z < hi)
        if alive is not None:
            sel &= alive
        for i in np.nonzero(sel)[0]:
            out[k, q[i], py[i], px[i]] += 1
    return out


class OracleRun:
    """One run advanced by the oracle: parameters, per-cell data, state, tallies."""

    def __init__(self, rp, state, E=None, ne_cells=None, dt=None, deposit=True):
        self.rp = rp
        self.p = make_params(rp, dt)
        nc = rp.ncells
        qmax = rp.species.qmax
        ip, nout = rp.species.ladder()
        self.rates = np.zeros(2 * qmax)
        lib().or_build_rates(ctypes.byref(self.p), _ptr(np.ascontiguousarray(ip, np.float64)),
                             _ptr(np.ascontiguousarray(nout, np.int32)), _ptr(self.rates))
        self.ratesr = np.zeros(2 * (qmax + 1))
        if rp.flags & F_RECOMB:
            lib().or_build_rates_rec(ctypes.byref(self.p), _ptr(self.ratesr))
        self.rates2 = np.zeros(4 * qmax)   # double by zone, then triple by zone
        if rp.flags & F_DOUBLE:
            lib().or_build_rates2(ctypes.byref(self.p), _ptr(np.ascontiguousarray(ip, np.float64)),
                                  _ptr(np.ascontiguousarray(nout, np.int32)), _ptr(self.rates2))
        self.ne = np.zeros(nc)
        self.zone = np.zeros(nc, dtype=np.int32)
        self.Bmag = np.zeros(nc)
        self.dlx = np.zeros(nc)
        self.dly = np.zeros(nc)
        nec = None if ne_cells is None else np.ascontiguousarray(ne_cells, np.float32)
        lib().or_setup_cells(ctypes.byref(self.p), _ptr(nec), rp.ne_in_cm3, rp.ne_out_cm3,
                             _ptr(self.ne), _ptr(self.zone), _ptr(self.Bmag), _ptr(self.dlx),
                             _ptr(self.dly))
        self.E = np.zeros(3 * nc) if E is None else np.ascontiguousarray(E, np.float64).reshape(-1)
        self.n = len(state["x"])
        self.set_state(state)
        self.status = np.zeros(self.n, dtype=np.uint32)
        self.tally = Tally()
        self.dep_count = np.zeros(nc, dtype=np.int64) if deposit else None
        self.dep_charge = np.zeros(nc, dtype=np.int64) if deposit else None
        self.events = np.zeros(self.n, dtype=np.uint8)
        self.guard = np.zeros(self.n, dtype=np.uint8)
        self.step_index = 0
        self.ne_mark_charge = None if self.dep_charge is None else self.dep_charge.copy()
        self.ne_mark_step = 0
        # first-passage times (Sec. III.D): step of each particle's last
        # ionisation from Q = 0 (-1: unknown, e.g. loaded as an ion), and the
        # ages of extracted ions by charge state
        self.birth = np.full(self.n, -1, dtype=np.int64)
        self.fptd_hist = np.zeros((qmax + 1, FPTD_BINS), dtype=np.int64)
        self.fptd_sum = np.zeros(qmax + 1, dtype=np.int64)

    def set_state(self, s):
        for k in ("x", "y", "z", "vx", "vy", "vz"):
            setattr(self, k, np.ascontiguousarray(s[k], dtype=np.float64).copy())
        self.q = np.ascontiguousarray(s["q"], dtype=np.int32).copy()

    def state(self):
        return {k: getattr(self, k) for k in ("x", "y", "z", "vx", "vy", "vz", "q")}

    def step(self, nsteps=1, accumulate_guard=False):
        """Advance nsteps; events/guard hold the last step (or the OR over steps)."""
        acc_ev = np.zeros(self.n, dtype=np.uint8)
        acc_g = np.zeros(self.n, dtype=np.uint8)
        for _ in range(nsteps):
            q_before = self.q.copy()
            lib().or_step(ctypes.byref(self.p), _ptr(self.rates), _ptr(self.rates2), _ptr(self.ratesr),
                          _ptr(self.ne), _ptr(self.zone),
                          _ptr(self.dlx), _ptr(self.dly), _ptr(self.E), self.n,
                          _ptr(self.x), _ptr(self.y), _ptr(self.z), _ptr(self.vx), _ptr(self.vy),
                          _ptr(self.vz), _ptr(self.q), _ptr(self.status), self.step_index,
                          _ptr(self.events), _ptr(self.guard), ctypes.byref(self.tally),
                          _ptr(self.dep_count), _ptr(self.dep_charge))
            self._first_passage(q_before)
            self.step_index += 1
            acc_ev |= self.events
            acc_g |= self.guard
        if accumulate_guard:
            self.events_acc, self.guard_acc = acc_ev, acc_g
        return self

    def _first_passage(self, q_before):
        """After a step: an extracted ion (it leaves with its charge state from
        before the step) adds its age since its birth; an atom ionised in this
        step is born now."""
        s = self.step_index
        ext = ((self.events & EV_EXTRACT) != 0) & (q_before >= 1) & (self.birth >= 0)
        for i in np.nonzero(ext)[0]:
            age = s - int(self.birth[i])
            self.fptd_hist[q_before[i], fptd_bin(age)] += 1
            self.fptd_sum[q_before[i]] += age
        born = (q_before == 0) & ((self.events & EV_IONIZE) != 0)
        self.birth[born] = s

    def update_ne(self):
        """Self-consistent electron density (Sec. II, charge neutrality): n_e
        of each cell becomes the ion charge density, w times the charge the
        cell collected since the previous update (or the start), averaged over
        the steps in between and divided by the cell volume; delta is then
        rebuilt from the new n_e."""
        if self.dep_charge is None:
            raise ValueError("update_ne needs the deposit")
        steps = self.step_index - self.ne_mark_step
        if steps <= 0:
            raise ValueError("update_ne: no step since the previous update")
        rp = self.rp
        vol = (2.0 * rp.R0 / rp.nx) * (2.0 * rp.R0 / rp.ny) * (rp.L / rp.nz)
        dq = (self.dep_charge - self.ne_mark_charge).astype(np.float64)
        self.ne = np.ascontiguousarray(rp.weight * dq / (steps * vol))
        lib().or_cell_delta(ctypes.byref(self.p), _ptr(self.ne), _ptr(self.zone), _ptr(self.Bmag),
                            _ptr(self.dlx), _ptr(self.dly))
        self.ne_mark_charge = self.dep_charge.copy()
        self.ne_mark_step = self.step_index

    def extracted(self):
        return np.array(self.tally.extracted[: self.rp.species.qmax + 1], dtype=np.int64)

    def lost(self):
        return np.array(self.tally.lost[: self.rp.species.qmax + 1], dtype=np.int64)
