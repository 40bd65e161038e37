"""GPU parity at the benchmark's full sizes, in the launch configuration
bench.py times, through the C ABI:

* the scaled run (Ar, 4e6 particles, 64x64x128 mesh, every process on,
  collisions between ions included) stepped by ecris_step as one graph per
  step (first on the load order, then sorted), compared element by element
  with the FP64 oracle stepping all 4e6 particles from the same state;
* two runs of the 64-run batched gas-flow scan (4.8e7 particles on the
  device), after the autotuner picked the batch's launch shape, each compared
  with the oracle stepping that run alone.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1507_03392_gb300 import inputs as I
from tests import parity as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def E():
    from paper_1507_03392_gb300 import ecris
    return ecris


def _clean(t):
    return t["q"] == 0 and t["events"] == 0 and t["pos"] == 0 and t["vel"] == 0


def test_scaled_run_full_size(E):
    wl = I.config_scaled()
    st = I.make_particles(wl)
    ne = I.make_ne_cells(wl)
    run = E.Run(wl.params, ne_cells=ne)
    run.load(st)
    # velocities to the FP32 rounding of the collision arithmetic (tabulated
    # A(s), FP32 logarithms), as in the collision kernels' own lock-step tests
    t, orc = P.lockstep(run, wl.params, st, 3, ne_cells=ne, vel_rel=5e-5)
    assert _clean(t), t["first_bad"]
    # every particle is compared; few lie near a decision surface, and fewer
    # still took the other side of one (explained by the oracle's probes)
    assert t["guarded_frac"] < 0.02 and t["accepted_frac"] < 0.01, t
    # (at dt = 1 ns three steps see a few tens of ionisations and no wall
    # hits; the collision count below shows the pairing ran at full size)
    assert t["events_seen"][2] > 0, t["events_seen"]
    d = run.diag()
    assert d["coulomb_collisions"] > 1e6
    run.close()


def test_batched_scan_full_size(E):
    wls = [I.config_oxygen_scan(i) for i in range(64)]
    states = [I.make_particles(wl) for wl in wls]
    b = E.Batch()
    hs = [b.add(wl.params, st) for wl, st in zip(wls, states)]
    b.autotune(trial_steps=4)
    checked = 0
    for i in (0, 63):
        wl, h = wls[i], hs[i]
        s0 = int(b.diag(h)["steps"])
        orc = O.OracleRun(wl.params, states[i])
        for s in range(s0, s0 + 2):
            g0 = b.state(h)
            orc.set_state({k: g0[k] for k in P.KEYS + ("q",)})
            orc.status[:] = np.where((g0["meta"] & (1 << 16)) != 0, 1, 0)
            orc.step_index = s
            orc.step(1)
            b.step(1)
            g1 = b.state(h)
            r = P.compare_step(wl.params, g1, orc, probes=P.Probes(wl.params, g0, s, orc))
            assert not (r["q"] or r["events"] or r["pos"] or r["vel"]), (i, s, r)
            checked += wl.n
    assert checked > 4 * 2e5
    b.close()
