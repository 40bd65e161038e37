"""GPU tests of the served form: a library thread keeps a batch of runs on the
device, admits queued requests as memory frees up and retires each run when
its extracted currents converge or it reaches its step cap.  A served result
must equal the same run stepped alone for the same number of steps."""
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


def specs():
    out = []
    rp = I.RunParams(nx=16, ny=16, nz=32, ne_in_cm3=2e12, ne_out_cm3=2e11, n0_cm3=1e11, dt=2e-8,
                     flags=I.F_ALL, seed=41)
    wl = I.Workload("a", rp, n=3001, steps=0, atom_fraction=0.5, ion_qmax_init=8, ion_T_eV=10.0,
                    atoms_fill_chamber=True, zone_box=(0.012, 0.15, 0.22))
    out.append((rp, I.make_particles(wl, seed=41), I.make_efield(rp, 2e3, -1e3)))
    rp = I.RunParams(species=I.OXYGEN, nx=8, ny=8, nz=16, ne_in_cm3=5e11, n0_cm3=3e11, dt=5e-9,
                     flags=I.F_ALL_NO_COULOMB, seed=42)
    wl = I.Workload("o", rp, n=5000, steps=0, atom_fraction=0.75, ion_qmax_init=6, ion_T_eV=5.0,
                    atoms_fill_chamber=True)
    out.append((rp, I.make_particles(wl, seed=42), None))
    rp = I.RunParams(species=I.KRYPTON, nx=8, ny=8, nz=16, ne_in_cm3=1e12, n0_cm3=1e11, dt=1e-8,
                     flags=I.F_ALL, seed=43)
    wl = I.Workload("k", rp, n=2000, steps=0, atom_fraction=0.25, ion_qmax_init=10, ion_T_eV=3.0,
                    atoms_fill_chamber=True)
    out.append((rp, I.make_particles(wl, seed=43), None))
    return out


def alone_diag(E, rp, st, Ef, steps):
    run = E.Run(rp, E=Ef)
    run.load(st)
    run.step(steps)
    d = run.diag()
    run.close()
    return d


def wait_all(srv, tickets, limit_s=180.0):
    t0 = time.time()
    while True:
        res = [srv.poll(t) for t in tickets]
        if all(r["state"] in (2, 3) for r in res):
            return res
        assert time.time() - t0 < limit_s, [r["state"] for r in res]
        time.sleep(0.01)


def check_equal(res, d):
    q1 = len(d["extracted"])
    assert np.array_equal(res["extracted"][:q1], d["extracted"])
    assert np.array_equal(res["lost"][:q1], d["lost"])
    assert res["ke_lost_eV"] == d["ke_lost_eV"]
    assert res["steps"] == d["steps"]


def test_served_results_equal_runs_alone(E):
    sp = specs()
    srv = E.Server(steps_per_tick=4)
    tickets = []
    for k, (rp, st, Ef) in enumerate(sp):
        # the first converges at its second window (any change is within a
        # tolerance of 1); the others can never meet min_events and hit the cap
        tol, min_ev = (1.0, 0) if k == 0 else (1e-3, 10**15)
        tickets.append(srv.submit(rp, st, E=Ef, window_steps=8, rel_tol=tol, min_events=min_ev,
                                  max_steps=24 + 8 * k))
    res = wait_all(srv, tickets)
    assert [r["state"] for r in res] == [E.REQ_DONE] * 3
    assert res[0]["converged"] and res[0]["steps"] == 16
    assert [r["steps"] for r in res[1:]] == [32, 40]
    for r, (rp, st, Ef) in zip(res, sp):
        check_equal(r, alone_diag(E, rp, st, Ef, r["steps"]))
        assert r["t_submit"] <= r["t_admit"] <= r["t_done"]
    s = srv.stats()
    assert s["done"] == 3 and s["queued"] == 0 and s["running"] == 0
    # each run is stepped up to one tick (4 steps) past the boundary it retired at
    used = sum(len(st["x"]) * r["steps"] for r, (_, st, _) in zip(res, sp))
    assert used <= s["ion_steps"] <= used + sum(len(st["x"]) * 4 for _, st, _ in sp)
    srv.close()


def busy_spec(seed):
    """hot ions in a dense plasma: many wall hits within a few tens of steps"""
    rp = I.RunParams(nx=16, ny=16, nz=32, ne_in_cm3=3e12, ne_out_cm3=3e11, n0_cm3=3e11, dt=3e-8,
                     Te_warm_eV=500.0, flags=I.F_ALL, seed=seed)
    wl = I.Workload("b", rp, n=8001, steps=0, atom_fraction=0.4, ion_qmax_init=8, ion_T_eV=60.0,
                    atoms_fill_chamber=True, zone_box=(0.02, 0.05, 0.29))
    return rp, I.make_particles(wl, seed=seed)


def test_served_self_consistent_ne_equals_run_alone(E):
    # n_e updated on the device after every 1 or 2 windows of 16 steps, with
    # no read-back in the request loop: the same as the run alone with
    # ecris_update_ne at the same steps, and not the same as without updates
    sp = [busy_spec(17), busy_spec(18)]
    srv = E.Server(steps_per_tick=4)
    tickets = [srv.submit(rp, st, window_steps=16, rel_tol=1e-3, min_events=10**15, max_steps=64, ne_windows=k + 1)
               for k, (rp, st) in enumerate(sp)]
    res = wait_all(srv, tickets)
    for k, (r, (rp, st)) in enumerate(zip(res, sp)):
        assert r["state"] == E.REQ_DONE and r["steps"] == 64
        run = E.Run(rp)
        run.load(st)
        for w in range(4):
            run.step(16)
            if (w + 1) % (k + 1) == 0:
                run.update_ne()
        check_equal(r, run.diag())
        run.close()
        d0 = alone_diag(E, rp, st, None, 64)   # the prescribed n_e throughout
        assert d0["lost"][1:].sum() > 100
        assert r["ke_lost_eV"] != d0["ke_lost_eV"]
    srv.close()


def test_budget_queues_in_arrival_order(E):
    sp = specs()
    rp, st, Ef = sp[1]
    need = E.ecris_run_bytes(len(st["x"]), rp.nx, rp.ny, rp.nz, 0)
    # room for one run at a time: the second waits for the first to retire
    srv = E.Server(hbm_budget=int(1.5 * need), steps_per_tick=8)
    ta = srv.submit(rp, st, window_steps=8, rel_tol=1e-3, min_events=10**15, max_steps=16)
    tb = srv.submit(rp, st, window_steps=8, rel_tol=1e-3, min_events=10**15, max_steps=24, seed=7)
    ra, rb = wait_all(srv, [ta, tb])
    assert ra["state"] == rb["state"] == E.REQ_DONE
    assert rb["t_admit"] >= ra["t_done"]
    check_equal(ra, alone_diag(E, rp, st, None, 16))
    rp7 = dataclasses.replace(rp, seed=7)
    check_equal(rb, alone_diag(E, rp7, st, None, 24))
    srv.close()


def test_rejects_invalid_requests(E):
    sp = specs()
    rp, st, Ef = sp[1]
    need = E.ecris_run_bytes(len(st["x"]), rp.nx, rp.ny, rp.nz, 0)
    srv = E.Server(hbm_budget=need // 2, steps_per_tick=4)
    with pytest.raises(E.EcrisError) as ei:
        srv.submit(rp, st, window_steps=8, max_steps=16)
    assert ei.value.status == E.ECRIS_ENOMEM and "budget" in str(ei.value)
    with pytest.raises(E.EcrisError) as ei:
        srv.submit(rp, st, window_steps=6, max_steps=12)   # not a multiple of the tick
    assert ei.value.status == E.ECRIS_EINVAL
    with pytest.raises(E.EcrisError):
        srv.poll(12345)
    srv.close()
