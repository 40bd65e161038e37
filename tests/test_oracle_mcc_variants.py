"""Pins of the oracle's opt-in processes of the collision block (Sec. II) and
the model variants of Secs. III.C and IV:

* double ionisation Q -> Q+2 and triple ionisation Q -> Q+3 beside Q -> Q+1
  (exact Markov chain with the closed-form rates);
* elastic ion-atom scattering, isotropic in the centre-of-mass frame (rate,
  kinematics, isotropy, competition with charge exchange);
* warm reflected atoms: ions neutralised at a wall come back at T_refl,
  atoms at T0;
* isotropic heating: the heating kick without the drift bias delta.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1507_03392_gb300 import inputs as I
from tests.test_oracle_mcc import _static, _uniform_params
from tests.test_oracle_rates import closed_form

QE = 1.602176634e-19
AMU = 1.66053906660e-27


def test_double_ionisation_matches_markov_chain():
    # single and double steps share one word: per step, Q -> Q+1 with
    # p k1/(k1+k2) and Q -> Q+2 with p k2/(k1+k2), p = 1 - exp(-n_e (k1+k2) dt);
    # k1 the Lotz-Maxwellian rate of P_Q, k2 = k2_factor times that of P_Q + P_{Q+1}
    rp = _uniform_params(flags=I.F_IONIZE | I.F_DOUBLE, dt=2e-7, k2_factor=0.3)
    n, S = 40000, 150
    r = O.OracleRun(rp, _static(n, 0, rp), deposit=False)
    ip, nout = rp.species.ladder()
    Te, ne = rp.Te_warm_eV, 1e18
    qm = rp.species.qmax
    k1 = np.array([closed_form(ip[q], nout[q], Te) for q in range(qm)])
    k2 = np.array([rp.k2_factor * closed_form(ip[q] + ip[q + 1], nout[q], Te) if q + 1 < qm else 0.0
                   for q in range(qm)])
    assert np.allclose(r.rates2[qm:2 * qm], k2, rtol=1e-6)
    assert not r.rates2[2 * qm:].any()            # no triple ionisation unless k3_factor > 0
    T = np.zeros((qm + 1, qm + 1))
    for q in range(qm):
        pt = 1 - math.exp(-ne * (k1[q] + k2[q]) * rp.dt)
        T[q, q] = 1 - pt
        T[q, q + 1] = pt * k1[q] / (k1[q] + k2[q])
        if q + 2 <= qm:
            T[q, q + 2] = pt * k2[q] / (k1[q] + k2[q])
    T[qm, qm] = 1.0
    r.step(S)
    got = np.bincount(r.q, minlength=qm + 1) / n
    want = np.linalg.matrix_power(T, S)[0]
    sig = np.sqrt(want * (1 - want) / n) + 1e-12
    assert np.all(np.abs(got - want) < 5 * sig + 1e-4)
    # without double ionisation the chain is the single-step one: a clear
    # difference at these parameters
    T1 = np.zeros_like(T)
    for q in range(qm):
        p1 = 1 - math.exp(-ne * k1[q] * rp.dt)
        T1[q, q], T1[q, q + 1] = 1 - p1, p1
    T1[qm, qm] = 1.0
    mean1 = (np.arange(qm + 1) * np.linalg.matrix_power(T1, S)[0]).sum()
    assert (np.arange(qm + 1) * got).sum() > mean1 + 0.2


def _chain(ks, ne, dt, qm):
    """one step's transition matrix for Q -> Q+1..Q+len(ks) sharing one word"""
    T = np.zeros((qm + 1, qm + 1))
    for q in range(qm):
        kq = [k[q] for k in ks]
        pt = 1 - math.exp(-ne * sum(kq) * dt)
        T[q, q] = 1 - pt
        for n, kn in enumerate(kq, start=1):
            if kn > 0:
                T[q, q + n] = pt * kn / sum(kq)
    T[qm, qm] = 1.0
    return T


def test_triple_ionisation_matches_markov_chain():
    # Q -> Q+1, Q+2, Q+3 share one word in proportion to k1, k2, k3; k3 =
    # k3_factor times the Lotz-Maxwellian rate of P_Q + P_{Q+1} + P_{Q+2}
    rp = _uniform_params(flags=I.F_IONIZE | I.F_DOUBLE, dt=2e-7, k2_factor=0.3, k3_factor=1.0)
    n, S = 40000, 150
    r = O.OracleRun(rp, _static(n, 0, rp), deposit=False)
    ip, nout = rp.species.ladder()
    Te, ne = rp.Te_warm_eV, 1e18
    qm = rp.species.qmax
    k1 = np.array([closed_form(ip[q], nout[q], Te) for q in range(qm)])
    k2 = np.array([rp.k2_factor * closed_form(ip[q] + ip[q + 1], nout[q], Te) if q + 1 < qm else 0.0
                   for q in range(qm)])
    k3 = np.array([rp.k3_factor * closed_form(ip[q] + ip[q + 1] + ip[q + 2], nout[q], Te) if q + 2 < qm else 0.0
                   for q in range(qm)])
    assert np.allclose(r.rates2[3 * qm:], k3, rtol=1e-6) and k3[qm - 2] == 0.0 and k3[qm - 3] > 0.0
    r.step(S)
    got = np.bincount(r.q, minlength=qm + 1) / n
    want = np.linalg.matrix_power(_chain([k1, k2, k3], ne, rp.dt, qm), S)[0]
    sig = np.sqrt(want * (1 - want) / n) + 1e-12
    assert np.all(np.abs(got - want) < 5 * sig + 1e-4)
    # the chain without the triple step is clearly rejected
    want2 = np.linalg.matrix_power(_chain([k1, k2], ne, rp.dt, qm), S)[0]
    sig2 = np.sqrt(want2 * (1 - want2) / n) + 1e-12
    assert np.max(np.abs(got - want2) / sig2) > 10


def test_double_ionisation_top_state():
    # from qmax - 1 only one electron is left: no double step there, and a
    # double step from qmax - 2 ends at qmax
    rp = I.RunParams(species=I.OXYGEN, B_ecr=100.0, ne_in_cm3=1e14, Te_warm_eV=3000.0,
                     flags=I.F_IONIZE | I.F_DOUBLE, k2_factor=1.0, dt=1e-5)
    qm = rp.species.qmax
    for q0 in (qm - 1, qm - 2):
        r = O.OracleRun(rp, _static(4000, q0, rp), deposit=False)
        assert r.rates2[qm + qm - 1] == 0.0 and r.rates2[qm + qm - 2] > 0.0
        r.step(1)
        ev = (r.events & O.EV_IONIZE) != 0
        assert ev.sum() > 200 and r.q.max() == qm
        if q0 == qm - 2:
            assert np.any(r.q[ev] == qm) and np.any(r.q[ev] == qm - 1)


def test_triple_ionisation_top_state():
    # a triple step needs three electrons: none from qmax - 2, and from
    # qmax - 3 it is the only way to reach qmax in one step
    rp = I.RunParams(species=I.OXYGEN, B_ecr=100.0, ne_in_cm3=1e14, Te_warm_eV=3000.0,
                     flags=I.F_IONIZE | I.F_DOUBLE, k2_factor=1.0, k3_factor=1.0, dt=1e-5)
    qm = rp.species.qmax
    r = O.OracleRun(rp, _static(4000, qm - 3, rp), deposit=False)
    assert r.rates2[2 * qm + qm + qm - 2] == 0.0 and r.rates2[2 * qm + qm + qm - 3] > 0.0
    r.step(1)
    assert r.q.max() == qm and np.any(r.q == qm - 1) and np.any(r.q == qm - 2)
    r = O.OracleRun(rp, _static(4000, qm - 2, rp), deposit=False)
    r.step(1)
    assert r.q.max() == qm


def _beam(rp, n, q, u):
    return _static(n, q, rp, v=(u, 0.0, 0.0))


def test_elastic_rate_kinematics_and_isotropy():
    # a monoenergetic beam (speed u along x) on background atoms at a tiny T0:
    # one step scatters 1 - exp(-n0 sigma_el Q v_rel dt) of it; with the atom
    # at rest the ion ends on the sphere |v' - u/2| = u/2, uniformly in angle
    rp = _uniform_params(flags=I.F_ELASTIC, n0_cm3=1e13, dt=2e-6, T0_eV=1e-6, sigma_el1_cm2=5e-15)
    n, u = 50000, 2.0e4
    M = rp.species.mass_amu * AMU
    for q in (1, 2, 4):
        r = O.OracleRun(rp, _beam(rp, n, q, u), deposit=False)
        r.step(1)
        ev = (r.events & O.EV_ELASTIC) != 0
        vrel = math.sqrt(u * u + 8 * rp.T0_eV * QE / (math.pi * M))
        pr = 1 - math.exp(-1e19 * 5e-19 * q * vrel * rp.dt)
        k = int(ev.sum())
        assert abs(k - n * pr) < 5 * math.sqrt(n * pr * (1 - pr)) + 1
        assert np.all(r.q == q) and np.all(r.vx[~ev] == u)
        d = np.stack([r.vx[ev] - u / 2, r.vy[ev], r.vz[ev]], axis=1) / (u / 2)
        rad = np.linalg.norm(d, axis=1)
        # the atom's thermal speed (about 2 m/s) blurs the sphere slightly
        assert np.all(np.abs(rad - 1) < 2e-3)
        assert np.all(np.abs(d.mean(axis=0)) < 5 / math.sqrt(3 * k))
        # energy in the lab frame: <|v'|^2> = u^2 / 2 for isotropic scattering
        v2 = (r.vx[ev] ** 2 + r.vy[ev] ** 2 + r.vz[ev] ** 2) / (u * u)
        assert abs(v2.mean() - 0.5) < 5 * v2.std() / math.sqrt(k)


def test_elastic_and_charge_exchange_share_the_word():
    # both on: any collision with probability 1 - exp(-n0 (sigma_cx + sigma_el)
    # v_rel dt), split in proportion to the cross sections; Q = 2 only scatters
    rp = _uniform_params(flags=I.F_ELASTIC | I.F_CX, n0_cm3=1e13, dt=2e-6, sigma_el1_cm2=5e-15)
    n, u = 60000, 1.5e4
    M = rp.species.mass_amu * AMU
    for q in (3, 2):
        r = O.OracleRun(rp, _beam(rp, n, q, u), deposit=False)
        r.step(1)
        vrel = math.sqrt(u * u + 8 * rp.T0_eV * QE / (math.pi * M))
        scx = 3e-19 * q if q != 2 else 0.0
        sel = 5e-19 * q
        pt = 1 - math.exp(-1e19 * (scx + sel) * vrel * rp.dt)
        for bit, frac in ((O.EV_CX, scx / (scx + sel)), (O.EV_ELASTIC, sel / (scx + sel))):
            k = int(((r.events & bit) != 0).sum())
            pr = pt * frac
            assert abs(k - n * pr) < 5 * math.sqrt(n * pr * (1 - pr)) + 1
        assert not np.any((r.events & O.EV_CX) & (r.events & O.EV_ELASTIC))


def _flange_hits(rp, n, q):
    """n particles on the axis just inside z = 0, moving onto the flange: each
    hits it in the first step and is re-emitted there."""
    st = _static(n, q, rp, v=(0.0, 0.0, -5.0e3))
    st["x"][:] = 0.0
    st["y"][:] = 0.0
    st["z"][:] = 1e-6
    return st


def test_warm_reflection_of_neutralised_ions():
    # re-emission by the cosine law at temperature T: normal speed sigma
    # sqrt(-2 ln U), so <v_n^2> = 2 sigma^2; tangential <v_t^2> = sigma^2
    # each, sigma^2 = kT/M.  Ions come back at T_refl, atoms at T0.
    rp = _uniform_params(flags=I.F_PUSH | I.F_RECYCLE, T_refl_eV=0.15, dt=1e-9)
    M = rp.species.mass_amu * AMU
    n = 40000
    for q, T in ((3, 0.15), (0, rp.T0_eV)):
        r = O.OracleRun(rp, _flange_hits(rp, n, q), deposit=False)
        r.step(1)
        assert np.all((r.events & O.EV_WALL) != 0) and np.all(r.q == 0)
        s2 = T * QE / M
        vn2 = (r.vz ** 2).mean() / (2 * s2)
        vt2 = ((r.vx ** 2 + r.vy ** 2) / 2).mean() / s2
        # relative standard deviations sqrt(2/n) and sqrt(1/n) (exponential and
        # chi-square-2 variables)
        assert abs(vn2 - 1) < 5 * math.sqrt(1 / n) and abs(vt2 - 1) < 5 * math.sqrt(1 / n)


def test_isotropic_heating_drops_delta():
    # a density ramp gives delta != 0 and a kick biased along delta; with the
    # isotropic-heating switch delta = 0 and the mean kick vanishes
    rp = I.RunParams(B_ecr=100.0, nx=12, ny=12, nz=6, flags=I.F_EIKICK | I.F_ISOHEAT, dt=1e-7)
    nc = rp.ncells
    iy = (np.arange(nc) // rp.nx) % rp.ny
    ne = (3e11 + 2e10 * iy).astype(np.float32)
    n = 40000
    st = _static(n, 3, rp)
    r = O.OracleRun(rp, st, ne_cells=ne, deposit=False)
    assert np.all(r.dlx == 0) and np.all(r.dly == 0)
    r.step(1)
    dv = np.stack([r.vx, r.vy, r.vz], axis=1)
    D = np.linalg.norm(dv, axis=1).mean()
    assert np.all(np.abs(dv.mean(axis=0)) < 5 * D / math.sqrt(3 * n))
    # the same run without the switch has delta along x and a biased mean kick
    r2 = O.OracleRun(I.RunParams(B_ecr=100.0, nx=12, ny=12, nz=6, flags=I.F_EIKICK, dt=1e-7), st, ne_cells=ne,
                     deposit=False)
    c = O.ngp_cells(rp, st["x"][:1], st["y"][:1], st["z"][:1])[0]
    assert r2.dlx[c] > 0


def test_recombination_rate_anchor_and_scaling():
    # Seaton's hydrogenic radiative-recombination rate: hydrogen at 1e4 K
    # has the textbook case-A coefficient 4.18e-13 cm^3/s (Seaton's
    # approximation lies within 2 % of it); the rate scales as
    # alpha(Z, T) = Z alpha(1, T / Z^2)
    lib = O.lib()
    a_h = lib.or_recomb_rate(1, 1e4 / 11604.518) * 1e6
    assert a_h == pytest.approx(4.18e-13, rel=0.03)
    for Z in (2, 5, 8, 18):
        for T in (5.0, 300.0, 3000.0):
            assert lib.or_recomb_rate(Z, T) == pytest.approx(Z * lib.or_recomb_rate(1, T / Z ** 2), rel=1e-12)
    # recombination is slow next to ionisation in the warm zone, faster in the cold periphery
    assert lib.or_recomb_rate(8, 1000.0) < lib.or_recomb_rate(8, 5.0)


def test_recombination_markov_chain():
    # ions at rest in cold, dense electrons: only Q -> Q-1, with per-step
    # probability 1 - exp(-n_e alpha_Q dt)
    rp = _uniform_params(flags=I.F_RECOMB, Te_warm_eV=5.0, Te_cold_eV=5.0, ne_in_cm3=1e14, ne_out_cm3=1e14,
                         dt=5e-5)
    n, S, q0 = 30000, 40, 8
    r = O.OracleRun(rp, _static(n, q0, rp), deposit=False)
    lib = O.lib()
    T = np.eye(q0 + 1)
    for q in range(1, q0 + 1):
        pr = 1 - math.exp(-1e20 * lib.or_recomb_rate(q, 5.0) * rp.dt)
        T[q, q], T[q, q - 1] = 1 - pr, pr
    r.step(S)
    got = np.bincount(r.q, minlength=q0 + 1)[: q0 + 1] / n
    want = np.linalg.matrix_power(T, S)[q0]
    sig = np.sqrt(want * (1 - want) / n) + 1e-12
    assert np.all(np.abs(got - want) < 5 * sig + 1e-4)
    assert want[q0] < 0.7          # the chain moved
    ev = (r.events & O.EV_RECOMB) != 0
    assert ev.sum() > 0


def test_recombination_and_ionisation_share_the_word():
    # both on: per step any change with p = 1 - exp(-n_e (k1 + kr) dt), up
    # with p k1/(k1+kr), down with p kr/(k1+kr)
    rp = _uniform_params(flags=I.F_RECOMB | I.F_IONIZE, Te_warm_eV=40.0, Te_cold_eV=40.0, ne_in_cm3=1e14,
                         ne_out_cm3=1e14, dt=2e-6)
    n, q0 = 60000, 3
    r = O.OracleRun(rp, _static(n, q0, rp), deposit=False)
    lib = O.lib()
    ip, nout = rp.species.ladder()
    k1 = closed_form(ip[q0], nout[q0], 40.0)
    kr = lib.or_recomb_rate(q0, 40.0)
    r.step(1)
    pt = 1 - math.exp(-1e20 * (k1 + kr) * rp.dt)
    for qq, frac in ((q0 + 1, k1 / (k1 + kr)), (q0 - 1, kr / (k1 + kr))):
        k = int((r.q == qq).sum())
        pr = pt * frac
        assert abs(k - n * pr) < 5 * math.sqrt(n * pr * (1 - pr)) + 1
