"""GPU parity of the on-axis field table (a computed or flat B0(z) profile
instead of the synthetic mirror), through the C ABI: lock-step with the
oracle, a batch and a served run against the same run alone, and invalid
tables."""
import dataclasses
import time

import numpy as np
import pytest

from oracle import oracle as O
from paper_1507_03392_gb300 import inputs as I
from tests import parity as P
from tests import test_gpu_parity as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def E():
    from paper_1507_03392_gb300 import ecris
    return ecris


def _flat_case(seed=4):
    rp, st, Ef = G.busy_case(seed=seed)
    rp = dataclasses.replace(rp, B_axial=I.flat_axial_profile(rp, n=257, flat=0.06))
    return rp, st, Ef


def test_lockstep_with_flat_profile(E):
    rp, st, Ef = _flat_case()
    run = E.Run(rp, E=Ef)
    run.load(st)
    t, orc = P.lockstep(run, rp, st, 60, E=Ef)
    assert t["q"] == 0 and t["events"] == 0 and t["pos"] == 0 and t["vel"] == 0, t["first_bad"]
    wall, ext, ion, cx = t["events_seen"]
    assert wall > 50 and ion > 15, t["events_seen"]
    run.close()


def test_batch_and_served_with_table_equal_run_alone(E):
    rp, st, Ef = _flat_case(seed=5)
    rp = dataclasses.replace(rp, flags=rp.flags | I.F_COULOMB)
    run = E.Run(rp, E=Ef)
    run.load(st)
    run.step(24)
    d = run.diag(grids=True)
    s = run.state()
    run.close()
    b = E.Batch()
    h = b.add(rp, st, E=Ef)
    b.step(24)
    db, sb = b.diag(h, grids=True), b.state(h)
    b.close()
    for key in ("extracted", "lost", "alive_by_q", "cell_charge"):
        assert np.array_equal(d[key], db[key]), key
    for key in ("x", "y", "z", "vx", "vy", "vz", "meta"):
        assert np.array_equal(s[key], sb[key]), key
    srv = E.Server(steps_per_tick=4)
    table = np.array(rp.B_axial)
    tk = srv.submit(rp, st, E=Ef, window_steps=8, rel_tol=1e-3, min_events=10 ** 15, max_steps=24)
    table[:] = 0.0          # the server holds its own copy
    t0 = time.time()
    while srv.poll(tk)["state"] not in (E.REQ_DONE, E.REQ_FAILED):
        assert time.time() - t0 < 120
        time.sleep(0.01)
    r = srv.poll(tk)
    srv.close()
    assert r["state"] == E.REQ_DONE and r["steps"] == 24
    q1 = len(d["extracted"])
    assert np.array_equal(r["extracted"][:q1], d["extracted"]) and r["ke_lost_eV"] == d["ke_lost_eV"]


def test_invalid_tables(E):
    rp = G.busy_case()[0]
    for bad in ((1.0, 0.5, 1.0), (1.0, float("nan"), 0.4, 1.0), (1.0, -0.1, 0.4, 1.0)):
        with pytest.raises(E.EcrisError) as ei:
            E.Run(dataclasses.replace(rp, B_axial=bad))
        assert ei.value.status == E.ECRIS_EINVAL
    # with a table the mirror's extremes are not needed
    run = E.Run(dataclasses.replace(rp, B_axial=(2.0, 0.4, 0.45, 1.1), B_inj=0.0, B_ext=0.0))
    run.close()
