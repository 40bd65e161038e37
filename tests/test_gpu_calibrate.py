"""GPU tests of calibration as a served workload (Sec. II: the weight and the
warm-electron temperature are adjusted until the converged plasma's gas flow
and coupled power meet targets): a job converges to targets it can reach, its
runs reproduce as plain requests with the same inputs, and invalid jobs are
rejected."""
import dataclasses
import time

import numpy as np
import pytest

from paper_1507_03392_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def E():
    from paper_1507_03392_gb300 import ecris
    return ecris


def _case():
    rp = I.RunParams(species=I.OXYGEN, nx=8, ny=8, nz=16, ne_in_cm3=3e12, ne_out_cm3=3e11, n0_cm3=1e11, dt=1e-7,
                     r_ap=0.02, flags=I.F_ALL_NO_COULOMB, seed=42, Te_warm_eV=1000.0)
    wl = I.Workload("c", rp, n=30000, steps=0, atom_fraction=0.5, ion_qmax_init=6, ion_T_eV=100.0,
                    atoms_fill_chamber=True)
    return rp, I.make_particles(wl, seed=42)


# every run is two windows of 128 steps: the rule (any change within a factor
# of 10) holds at the second window boundary
RULE = dict(window_steps=128, rel_tol=10.0, min_events=1, max_steps=256)


def _wait(srv, fn, key, limit=300.0):
    """Poll fn(key) until the request or job is done or failed."""
    t0 = time.time()
    while True:
        r = fn(key)
        if r["state"] in (2, 3):
            return r
        assert time.time() - t0 < limit
        time.sleep(0.02)


def test_calibration_meets_reachable_targets(E):
    rp, st = _case()
    srv = E.Server(steps_per_tick=32)
    tk = srv.submit(rp, st, **RULE)
    base = _wait(srv, srv.poll, tk)
    assert base["state"] == E.REQ_DONE and base["steps"] == 256
    F0, P0 = base["flow_per_s"], base["power_window_W"]
    assert F0 > 0 and P0 > 0
    # twice the flow (w alone reaches it) at 20 % more energy per particle (T_ew)
    Ft, Pt = 2.0 * F0, 2.4 * P0
    job = srv.calibrate(rp, st, Ft, Pt, tol=0.05, max_iter=8, **RULE)
    res = _wait(srv, srv.calib_poll, job)
    assert res["state"] == E.REQ_DONE and res["met"], res
    k = res["iterations"]
    assert 2 <= k <= 8
    assert res["weight"][0] == rp.weight and res["Te_warm_eV"][0] == rp.Te_warm_eV
    assert res["flow_per_s"][0] == F0 and res["power_W"][0] == P0   # the first run is the base run
    assert abs(res["flow_per_s"][-1] / Ft - 1) <= 0.05 and abs(res["power_W"][-1] / Pt - 1) <= 0.05
    assert res["weight"][-1] == pytest.approx(2.0 * rp.weight, rel=0.1)
    assert res["Te_warm_eV"][-1] > rp.Te_warm_eV
    # the last run, served as a plain request with the same inputs, gives the same outputs
    rp2 = dataclasses.replace(rp, Te_warm_eV=float(res["Te_warm_eV"][-1]), weight=float(res["weight"][-1]))
    again = _wait(srv, srv.poll, srv.submit(rp2, st, weight=float(res["weight"][-1]), **RULE))
    assert again["flow_per_s"] == res["flow_per_s"][-1] and again["power_window_W"] == res["power_W"][-1]
    srv.close()
    # the FP64 oracle over the same run: its last window's gas flow and power
    F_o, P_o, n_out, n_left = oracle_window_outputs(rp2, st, RULE["window_steps"], RULE["max_steps"])
    print(f"\n[calibration, final run] gas flow GPU {res['flow_per_s'][-1]:.6e} / oracle {F_o:.6e} per s "
          f"({n_out} particles out in the window); power GPU {res['power_W'][-1]:.6e} / oracle {P_o:.6e} W "
          f"({n_left} ions left)")
    assert abs(res["flow_per_s"][-1] - F_o) <= max(0.01, 3.0 / np.sqrt(max(n_out, 1))) * F_o
    assert abs(res["power_W"][-1] - P_o) <= max(0.01, 3.0 / np.sqrt(max(n_left, 1))) * P_o


def oracle_window_outputs(rp, st, window, steps):
    """Gas flow and power of the oracle run's last window (Sec. II: the two
    outputs of the model): the flow is the weight times the particles (ions
    and atoms) that went out through the aperture in the window, per second;
    the power is the weight times the energy the ions that left in the window
    carried out -- kinetic energy, the ionisation energies of their charge
    state, and 3/2 T_ew for each of their electrons -- per second."""
    from oracle import oracle as O
    orc = O.OracleRun(rp, st, deposit=False)
    orc.step(steps - window)
    ext0, lost0, ke0 = orc.extracted().copy(), orc.lost().copy(), orc.tally.ke_lost_eV
    orc.step(window)
    d_ext, d_lost = orc.extracted() - ext0, orc.lost() - lost0
    t_win = window * rp.dt
    flow = rp.weight * float(d_ext.sum()) / t_win
    ip, _ = rp.species.ladder()
    e_eV = orc.tally.ke_lost_eV - ke0
    ip_cum = np.concatenate([[0.0], np.cumsum(ip)])
    for q in range(1, rp.species.qmax + 1):
        e_eV += float(d_ext[q] + d_lost[q]) * (ip_cum[q] + 1.5 * q * rp.Te_warm_eV)
    power = rp.weight * e_eV * 1.602176634e-19 / t_win
    return flow, power, int(d_ext.sum()), int((d_ext[1:] + d_lost[1:]).sum())


def test_calibration_rejects_invalid_jobs(E):
    rp, st = _case()
    srv = E.Server(steps_per_tick=32)
    for kw in (dict(flow_target=0.0, power_target_W=1.0), dict(flow_target=1.0, power_target_W=-1.0),
               dict(flow_target=1.0, power_target_W=1.0, tol=0.0),
               dict(flow_target=1.0, power_target_W=1.0, max_iter=0),
               dict(flow_target=1.0, power_target_W=1.0, max_iter=33)):
        with pytest.raises(E.EcrisError) as ei:
            srv.calibrate(rp, st, **kw, **RULE)
        assert ei.value.status == E.ECRIS_EINVAL
    with pytest.raises(E.EcrisError):
        srv.calib_poll(99)
    srv.close()
