"""Pins of the oracle's Monte-Carlo collision block (Sec. II): step-wise
ionisation from the cell's n_e and T_e, charge exchange with the neutral
background, and the electron-ion heating kick with the delta stencil."""
import math
import os

import numpy as np
import pytest
from scipy.linalg import expm

from oracle import oracle as O
from paper_1507_03392_gb300 import inputs as I

QE = 1.602176634e-19
AMU = 1.66053906660e-27
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _static(n, q, rp, v=None):
    """n particles at rest (or with velocity v) at one point in the middle of a cell."""
    x0, y0, z0 = 0.0011, -0.0007, 0.1523
    st = {"x": np.full(n, x0), "y": np.full(n, y0), "z": np.full(n, z0),
          "vx": np.zeros(n), "vy": np.zeros(n), "vz": np.zeros(n),
          "q": np.full(n, q, dtype=np.int32)}
    if v is not None:
        st["vx"][:], st["vy"][:], st["vz"][:] = v
    return st


def _uniform_params(**kw):
    base = dict(ne_in_cm3=1e12, ne_out_cm3=1e12, Te_warm_eV=1000.0, Te_cold_eV=1000.0)
    base.update(kw)
    return I.RunParams(**base)


def test_zero_d_ionisation_matches_markov_chain_and_rate_equations():
    rp = _uniform_params(flags=I.F_IONIZE, dt=2e-7)
    n, S = 40000, 200
    r = O.OracleRun(rp, _static(n, 0, rp), deposit=False)
    lam = 1e18 * r.rates[18:36] * rp.dt       # warm-zone rates, n_e in m^-3
    p = 1 - np.exp(-lam)
    T = np.zeros((19, 19))
    for qq in range(18):
        T[qq, qq], T[qq, qq + 1] = 1 - p[qq], p[qq]
    T[18, 18] = 1.0
    r.step(S)
    got = np.bincount(r.q, minlength=19) / n
    want = np.linalg.matrix_power(T, S)[0]
    sig = np.sqrt(want * (1 - want) / n) + 1e-12
    assert np.all(np.abs(got - want) < 5 * sig + 1e-4)
    # continuous rate equations dN_Q/dt = k_{Q-1} n_e N_{Q-1} - k_Q n_e N_Q agree to O(lambda)
    G = np.zeros((19, 19))
    for qq in range(18):
        G[qq, qq] -= lam[qq] / rp.dt
        G[qq + 1, qq] += lam[qq] / rp.dt
    cont = expm(G * S * rp.dt)[:, 0]
    mean_got = (np.arange(19) * got).sum()
    mean_cont = (np.arange(19) * cont).sum()
    assert mean_got == pytest.approx(mean_cont, rel=0.02)


def test_ionisation_uses_the_cold_rate_outside_the_zone():
    # B_ecr below every |B| in the chamber: all cells are cold-electron cells
    rp = _uniform_params(flags=I.F_IONIZE, dt=1e-6, B_ecr=0.01, Te_cold_eV=20.0)
    n = 30000
    r = O.OracleRun(rp, _static(n, 0, rp), deposit=False)
    assert r.zone.sum() == 0
    r.step(1)
    pr = 1 - math.exp(-1e18 * r.rates[0] * rp.dt)
    k = (r.q == 1).sum()
    assert abs(k - n * pr) < 5 * math.sqrt(n * pr * (1 - pr)) + 1


def test_charge_exchange_zero_d():
    rp = _uniform_params(flags=I.F_CX, n0_cm3=1e12, dt=1e-5)
    n = 40000
    for q in (5, 2, 1):
        r = O.OracleRun(rp, _static(n, q, rp), deposit=False)
        r.step(1)
        M = 40 * AMU
        vrel = math.sqrt(8 * rp.T0_eV * QE / (math.pi * M))
        pr = 1 - math.exp(-1e18 * 3e-19 * q * vrel * rp.dt)
        ev = (r.events & O.EV_CX) != 0
        if q == 2:
            assert ev.sum() == 0 and np.all(r.q == 2)   # energetically forbidden
            continue
        k = ev.sum()
        assert abs(k - n * pr) < 5 * math.sqrt(n * pr * (1 - pr)) + 1
        speed = np.sqrt(r.vx ** 2 + r.vy ** 2 + r.vz ** 2)
        if q == 5:
            # Q -> Q-1 and an isotropic kick carrying half of the 10 eV release
            assert np.all(r.q[ev] == 4) and np.all(r.q[~ev] == 5)
            dv = math.sqrt(2 * 5.0 * QE / M)
            assert np.allclose(speed[ev], dv, rtol=1e-12)
            assert abs(r.vz[ev].mean()) < 5 * dv / math.sqrt(3 * k)
        else:
            assert np.all(r.q == 1)                    # resonant: the ion stays Q=1
            assert np.all(speed[~ev] == 0.0)


def test_resonant_charge_exchange_gives_thermal_ions():
    rp = _uniform_params(flags=I.F_CX, n0_cm3=1e14, dt=1e-4)
    n = 40000
    r = O.OracleRun(rp, _static(n, 1, rp), deposit=False)
    r.step(1)
    ev = (r.events & O.EV_CX) != 0
    assert ev.sum() > 10000
    s2 = rp.T0_eV * QE / (40 * AMU)
    for comp in (r.vx[ev], r.vy[ev], r.vz[ev]):
        assert comp.var() == pytest.approx(s2, rel=0.05)
        assert abs(comp.mean()) < 5 * math.sqrt(s2 / ev.sum())


def _kick(rp, q=2, n=20000):
    r = O.OracleRun(rp, _static(n, q, rp), deposit=False)
    r.step(1)
    return r, np.stack([r.vx, r.vy, r.vz], axis=1)


def test_kick_amplitude_golden_value():
    row = np.loadtxt(os.path.join(GOLDEN, "ei_kick_D.txt"))
    ne, Te, q, mass, dt, lnl, D = row
    rp = _uniform_params(flags=I.F_EIKICK, ne_in_cm3=ne, ne_out_cm3=ne, Te_warm_eV=Te,
                         Te_cold_eV=Te, dt=dt, lnL_ei=lnl)
    assert rp.species.mass_amu == mass
    r, dv = _kick(rp, q=int(q), n=2000)
    assert np.allclose(np.linalg.norm(dv, axis=1), D, rtol=1e-5)


def test_kick_scalings_and_isotropy():
    base = dict(flags=I.F_EIKICK, dt=1e-9)
    r0, dv0 = _kick(_uniform_params(**base))
    D0 = np.linalg.norm(dv0, axis=1)
    assert np.allclose(D0, D0[0], rtol=1e-12)     # |dV| = D for every ion (delta = 0)
    # isotropic direction: zero mean, <dv_z^2> = D^2/3
    assert np.abs(dv0.mean(axis=0)).max() < 5 * D0[0] / math.sqrt(3 * len(D0))
    assert (dv0[:, 2] ** 2).mean() == pytest.approx(D0[0] ** 2 / 3, rel=0.05)
    D0 = D0[0]

    def D(**kw):
        args = dict(base)
        args.update(kw)
        q = args.pop("q", 2)
        return np.linalg.norm(_kick(_uniform_params(**args), q=q, n=4)[1][0])

    assert D(ne_in_cm3=2e12, ne_out_cm3=2e12) ** 2 == pytest.approx(2 * D0 ** 2, rel=1e-9)
    assert D(q=4) ** 2 == pytest.approx(4 * D0 ** 2, rel=1e-9)             # Q^2
    assert D(ei_charge_power=1, q=4) ** 2 == pytest.approx(0.5 * D(ei_charge_power=1, q=8) ** 2, rel=1e-9)
    assert D(dt=2e-9) ** 2 == pytest.approx(2 * D0 ** 2, rel=1e-9)
    assert D(lnL_ei=34.0) ** 2 == pytest.approx(2 * D0 ** 2, rel=1e-9)
    assert D(Te_warm_eV=250.0, Te_cold_eV=250.0) ** 2 == pytest.approx(2 * D0 ** 2, rel=1e-9)
    oxy = dict(base, species=I.OXYGEN)
    ratio = (D(**oxy) / D0) ** 2
    assert ratio == pytest.approx((40.0 / 16.0) ** 2, rel=1e-9)           # 1/M^2


def test_kick_direction_follows_delta():
    # a density ramp in y gives delta along +x (printed stencil); the mean kick
    # points along delta and |dV| stays D
    rp = I.RunParams(flags=I.F_EIKICK, B_ecr=100.0, dt=1e-9, nx=16, ny=16, nz=8)
    nc = rp.ncells
    iy = (np.arange(nc) // rp.nx) % rp.ny
    ne_cells = (1e11 * (1.0 + 2.0 * iy)).astype(np.float32)
    st = _static(200000, 3, rp)
    r = O.OracleRun(rp, st, ne_cells=ne_cells, deposit=False)
    c = 0
    gx = (st["x"][0] + rp.R0) / (2 * rp.R0 / rp.nx)
    gy = (st["y"][0] + rp.R0) / (2 * rp.R0 / rp.ny)
    gz = st["z"][0] / (rp.L / rp.nz)
    c = (int(gz) * rp.ny + int(gy)) * rp.nx + int(gx)
    assert r.dlx[c] > 0.01 and abs(r.dly[c]) < 1e-12
    r.step(1)
    dv = np.stack([r.vx, r.vy, r.vz], axis=1)
    D = np.linalg.norm(dv, axis=1)
    assert np.allclose(D, D[0], rtol=1e-12)
    # for an isotropic unit R and |delta| < 1 the mean of (R+delta)/|R+delta|
    # is exactly (2/3) delta
    m = dv.mean(axis=0) / D[0]
    sig = math.sqrt(1 / (3 * len(D)))
    assert m[0] == pytest.approx(2 / 3 * r.dlx[c], abs=5 * sig)
    assert m[1] == pytest.approx(2 / 3 * r.dly[c], abs=5 * sig)
    assert abs(m[2]) < 5 * sig
