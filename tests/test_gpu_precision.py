"""Precision report of the FP32 CUDA path (GPU).

The push and the MCC block run in FP32; the diagnostics accumulate in 64-bit
integers (extracted / lost counts, the time-summed deposit grids) or 64-bit
fixed point (the energy carried to the walls, in micro-eV).  For a set of
scan-shaped runs this test states, per run:

* the error of each result of a free run against the FP64 oracle run from the
  same state with the same counter-based random words (charge-state
  distribution, extracted and lost counts, energy to the walls, collision
  count, time-summed deposit, positions of the particles with identical
  integer histories);
* what FP32 accumulation of the same per-step increments would have cost
  against the 64-bit accumulators the library keeps.

`python -m pytest tests/test_gpu_precision.py -m gpu -s` prints the table; the
asserted bounds are the parity bar (ensemble charge-state distribution and
extracted currents within 1 % relative of the oracle).
"""
import dataclasses

import numpy as np
import pytest

from oracle import oracle as O
from paper_1507_03392_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def E():
    from paper_1507_03392_gb300 import ecris
    return ecris


def workloads():
    """(name, workload, E grid, steps): the small plain run as specified, and
    scan-shaped runs long enough (tens of microseconds) for ionisation,
    charge exchange, losses and extraction to change the ensemble."""
    out = []
    wl = I.config_small(n=10_000, steps=1000)
    out.append(("Ar 1e4, 32x32x64, dt 1e-9 s, no n0, no ion-ion (plain run)", wl, None, 1000))
    wl = I.config_oxygen_scan(40, n=20_000)
    wl.params = dataclasses.replace(wl.params, dt=1e-8)
    out.append((f"O 2e4, n0 {wl.params.n0_cm3:.1e} cm^-3, dt 1e-8 s, no ion-ion (gas-flow scan run)", wl, None,
                2000))
    wl = I.config_power_scan(7, n=20_000)
    wl.params = dataclasses.replace(wl.params, dt=1e-8)
    p = wl.params
    out.append((f"Ar 2e4, ne {p.ne_in_cm3:.1e} cm^-3, Tew {p.Te_warm_eV:.0f} eV, dt 1e-8 s, all processes "
                "(power scan run)", wl, None, 2000))
    rp = I.RunParams(species=I.KRYPTON, nx=32, ny=32, nz=64, ne_in_cm3=1e12, n0_cm3=1e11, flags=I.F_ALL,
                     seed=5007, dt=1e-8)
    wl = I.Workload("kr", rp, n=10_000, steps=2000, atom_fraction=0.5, ion_qmax_init=12, ion_T_eV=5.0,
                    atoms_fill_chamber=True)
    out.append(("Kr 1e4, dt 1e-8 s, all processes (served-stream run)", wl, None, 2000))
    return out


def rel(a, b):
    a, b = float(a), float(b)
    return abs(a - b) / max(abs(b), 1e-300) if (a or b) else 0.0


def fp32_long(xs, total_steps=10_000_000):
    """Relative error of accumulating a run's per-step increments in FP32
    over total_steps steps (the increments repeated), against the exact sum."""
    xs = np.asarray(xs, dtype=np.float64)
    reps = max(1, total_steps // len(xs))
    tiled = np.tile(xs, reps)
    exact = tiled.sum(dtype=np.float64)
    acc = np.cumsum(tiled.astype(np.float32), dtype=np.float32)[-1]
    return rel(acc, exact), reps * len(xs)


@pytest.mark.parametrize("k", range(4))
def test_precision_against_oracle(E, k, capsys):
    name, wl, Ef, steps = workloads()[k]
    rp = wl.params
    st = I.make_particles(wl)
    ne = I.make_ne_cells(wl)
    run = E.Run(rp, E=Ef, ne_cells=ne)
    run.load(st)
    qe = 1.602176634e-19
    charges = np.arange(rp.species.qmax + 1, dtype=np.float64)
    prev_ext = np.zeros(rp.species.qmax + 1, np.int64)
    prev_ke = 0.0
    prev_cnt = None
    dq, dke, dcnt = [], [], []
    busiest = None
    for _ in range(steps):
        run.step(1)
        d = run.diag(grids=True)
        if busiest is None:
            busiest = int(np.argmax(d["cell_count"]))
            prev_cnt = np.uint64(0)
        dq.append(float((charges * (d["extracted"] - prev_ext)).sum()) * qe * rp.weight)
        dke.append(d["ke_lost_eV"] - prev_ke)
        dcnt.append(float(d["cell_count"][busiest] - prev_cnt))
        prev_ext, prev_ke, prev_cnt = d["extracted"].copy(), d["ke_lost_eV"], d["cell_count"][busiest]
    g = run.state()
    run.close()

    orc = O.OracleRun(rp, st, E=Ef, ne_cells=ne)
    orc.step(steps, accumulate_guard=True)
    alive_o = np.bincount(orc.q, minlength=rp.species.qmax + 1)[: rp.species.qmax + 1]
    alive_g = d["alive_by_q"]
    big = alive_o >= 1000
    csd_err = max(rel(alive_g[q], alive_o[q]) for q in np.nonzero(big)[0])
    csd_l1 = np.abs(alive_g - alive_o).sum() / alive_o.sum()
    ext_o, lost_o = orc.extracted(), orc.lost()
    q_ext_g = float((charges * d["extracted"]).sum())
    q_ext_o = float((charges * ext_o).sum())
    ke_err = rel(d["ke_lost_eV"], orc.tally.ke_lost_eV)
    coul_err = rel(d["coulomb_collisions"], orc.tally.coulomb_pairs)
    dep_err = np.abs(d["cell_count"].astype(np.float64) - orc.dep_count).sum() / max(1, orc.dep_count.sum())
    ok = (orc.guard_acc & O.G_SINGLE) == 0
    same = ok & (g["q"] == orc.q)
    pos_err = max(float((np.abs(g[c][same] - getattr(orc, c)[same]) / s).max())
                  for c, s in (("x", rp.R0), ("y", rp.R0), ("z", rp.L)))
    # FP32 accumulation of the same per-step increments over a production-length run
    q32_err, nlong = fp32_long(dq)
    ke32_err, _ = fp32_long(dke)
    cnt32_err, _ = fp32_long(dcnt)
    with capsys.disabled():
        print(f"\n[{name}] {steps} steps, {len(st['x'])} particles")
        print(f"  vs FP64 oracle: CSD max rel {csd_err:.2e} (Q with >= 1000), CSD L1 {csd_l1:.2e}, "
              f"extracted charge rel {rel(q_ext_g, q_ext_o):.2e} ({int(d['extracted'].sum())} vs "
              f"{int(ext_o.sum())} events), lost {int(d['lost'].sum())} vs {int(lost_o.sum())}, "
              f"wall energy rel {ke_err:.2e}, collisions rel {coul_err:.2e}, deposit L1 {dep_err:.2e}, "
              f"identical histories {same.mean():.4f}, position max rel {pos_err:.2e}")
        print(f"  FP32 accumulation instead, over {nlong} steps of these increments: extracted charge rel "
              f"{q32_err:.2e}, wall energy rel {ke32_err:.2e}, busiest cell's deposit time sum rel {cnt32_err:.2e} "
              f"(the library's 64-bit integer / fixed-point accumulators: exact / 1 micro-eV per event)")
    # the bar: every well-populated charge state within 1 % (the L1 sum over
    # all states, sparse ones included, is reported above)
    assert csd_err < 1e-2
    if ext_o.sum() >= 100:
        assert rel(q_ext_g, q_ext_o) < 1e-2
    if not rp.flags & I.F_COULOMB:
        if lost_o.sum() >= 100:
            assert rel(d["lost"].sum(), lost_o.sum()) < 1e-2
        # without collisions between ions no FP32 difference feeds back into
        # other particles: losses, energies and positions stay at rounding
        # level (with them, a pairing that differs after a guarded cell
        # crossing changes the partners' velocities and the difference
        # spreads; those results are reported, not bounded)
        assert ke_err < 1e-2
        assert pos_err < 1e-5
