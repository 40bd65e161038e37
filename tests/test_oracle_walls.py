"""Pins of the oracle's wall and aperture bookkeeping and deposition (Sec. II):
cosine-law diffuse re-emission with Maxwell-Boltzmann velocities at the gas
temperature, extraction through the round aperture with reinjection at the gas
inlet (constant particle number), and NGP counts of number and charge."""
import ctypes
import math

import numpy as np
import pytest
from scipy import stats

from oracle import oracle as O
from paper_1507_03392_gb300 import inputs as I

QE = 1.602176634e-19
AMU = 1.66053906660e-27


def test_cosine_law_sampler_moments():
    sigma = 250.0
    n = 60000
    nrm = np.array([0.0, 0.0, 1.0])
    e1 = np.array([1.0, 0.0, 0.0])
    e2 = np.array([0.0, 1.0, 0.0])
    vs = np.zeros((n, 3))
    ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    for i in range(n):
        w = O.philox([i, 0, 2, 0], [99, 0])
        v = np.zeros(3)
        O.lib().or_emit(sigma, ptr(nrm), ptr(e1), ptr(e2), ptr(w), ptr(v))
        vs[i] = v
    vn = vs[:, 2]
    assert np.all(vn > 0)
    # flux-weighted Maxwellian: <v_n> = sigma sqrt(pi/2), <v_n^2> = 2 sigma^2
    assert vn.mean() == pytest.approx(sigma * math.sqrt(math.pi / 2), rel=0.01)
    assert (vn ** 2).mean() == pytest.approx(2 * sigma ** 2, rel=0.02)
    assert vs[:, 0].var() == pytest.approx(sigma ** 2, rel=0.02)
    assert vs[:, 1].var() == pytest.approx(sigma ** 2, rel=0.02)
    # cosine law: the polar angle obeys P(cos theta <= c) = c^2
    c = vn / np.linalg.norm(vs, axis=1)
    assert stats.kstest(c, lambda t: np.clip(t, 0, 1) ** 2).pvalue > 1e-3


def _busy_params(**kw):
    # hot ions, strong heating and short steps: many wall hits and extractions
    base = dict(nx=16, ny=16, nz=32, ne_in_cm3=1e12, ne_out_cm3=2e11, dt=2e-8,
                flags=I.F_ALL_NO_COULOMB, n0_cm3=1e11)
    base.update(kw)
    return I.RunParams(**base)


def _busy_state(rp, n, seed=4):
    wl = I.Workload("busy", rp, n=n, steps=0, atom_fraction=0.3, ion_qmax_init=6,
                    ion_T_eV=40.0, atoms_fill_chamber=True)
    return I.make_particles(wl, seed=seed)


def test_recycling_keeps_particles_inside_and_neutralises_leavers():
    rp = _busy_params()
    st = _busy_state(rp, 4000)
    r = O.OracleRun(rp, st)
    total_ev = 0
    for _ in range(60):
        qprev = r.q.copy()
        r.step(1)
        rr = np.hypot(r.x, r.y)
        assert np.all(rr <= rp.R0) and np.all(r.z >= 0) and np.all(r.z <= rp.L)
        left = (r.events & (O.EV_WALL | O.EV_EXTRACT)) != 0
        assert np.all(r.q[left] == 0)
        total_ev += left.sum()
        # reinjected particles start at the gas inlet
        ex = (r.events & O.EV_EXTRACT) != 0
        assert np.allclose(r.x[ex], rp.inlet[0]) and np.allclose(r.z[ex], rp.inlet[2])
    assert total_ev > 20
    assert r.lost().sum() > 0
    assert r.tally.ke_lost_eV > 0


def test_without_recycling_alive_plus_lost_plus_extracted_is_n():
    rp = _busy_params(flags=I.F_ALL_NO_COULOMB & ~I.F_RECYCLE)
    n = 3000
    r = O.OracleRun(rp, _busy_state(rp, n))
    for _ in range(40):
        r.step(1)
        alive = int((r.status & 1 == 0).sum())
        assert alive + r.extracted().sum() + r.lost().sum() == n
    assert alive < n


def test_extraction_only_through_the_aperture():
    # ions fired straight at the extraction flange: those inside r_ap leave
    # through the aperture, the others hit the flange
    rp = I.RunParams(flags=I.F_PUSH | I.F_RECYCLE, B_inj=1e-9, B_min=0.0, B_ext=1e-9, B_hex=0.0,
                     dt=1e-7)
    n = 400
    rr = np.linspace(0.0, 0.02, n)
    st = {"x": rr.copy(), "y": np.zeros(n), "z": np.full(n, rp.L - 1e-4),
          "vx": np.zeros(n), "vy": np.zeros(n), "vz": np.full(n, 5000.0), "q": np.full(n, 3)}
    r = O.OracleRun(rp, st)
    r.step(1)
    ex = (r.events & O.EV_EXTRACT) != 0
    wall = (r.events & O.EV_WALL) != 0
    assert np.all(ex == (rr < rp.r_ap))
    assert np.all(wall == (rr >= rp.r_ap))
    assert r.extracted()[3] == ex.sum() and r.lost()[3] == wall.sum()
    ke = 0.5 * 40 * AMU * 5000.0 ** 2 / QE
    assert r.tally.ke_lost_eV == pytest.approx(n * ke, rel=1e-12)


def test_deposit_matches_brute_force_histogram():
    rp = _busy_params()
    st = _busy_state(rp, 3000, seed=9)
    r = O.OracleRun(rp, st)
    want_c = np.zeros(rp.ncells, dtype=np.int64)
    want_q = np.zeros(rp.ncells, dtype=np.int64)
    dx, dy, dz = 2 * rp.R0 / rp.nx, 2 * rp.R0 / rp.ny, rp.L / rp.nz
    for _ in range(20):
        r.step(1)
        ix = np.clip(np.floor((r.x + rp.R0) / dx).astype(int), 0, rp.nx - 1)
        iy = np.clip(np.floor((r.y + rp.R0) / dy).astype(int), 0, rp.ny - 1)
        iz = np.clip(np.floor(r.z / dz).astype(int), 0, rp.nz - 1)
        c = (iz * rp.ny + iy) * rp.nx + ix
        want_c += np.bincount(c, minlength=rp.ncells)
        want_q += np.bincount(c, weights=r.q, minlength=rp.ncells).astype(np.int64)
    assert np.array_equal(r.dep_count, want_c)
    assert np.array_equal(r.dep_charge, want_q)
