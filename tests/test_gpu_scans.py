"""Per-run parity of the two batched scans with the FP64 oracle (GPU).

The gas-flow scan asks for each run's charge-state currents against the FP64
oracle, and the microwave-power scan for the error of FP32 against FP64
accumulation in each run (Sec. II: the model's output is the charge-state
distribution of the extracted ions; Sec. III: the currents).  Here runs spread
over each scan's parameter range are stepped together in one batch, the way
the benchmark steps the scans, at 2e4 particles each so that the oracle can
follow every run:

* gas-flow scan: eight of the 64 runs (n0 from 3e9 to 3e11 cm^-3), autotuned
  launch shape; each run's extracted and in-chamber counts by charge state
  against its oracle run, within max(1 % of the oracle's count,
  3 sqrt(N_gpu + N_oracle)), the bound for two runs whose histories part after
  a flip (see test_gpu_ensemble.py);
* power scan: six of the 128 runs (n_e 5e10-2e12 cm^-3, T_ew 0.3-3 keV, every
  process with collisions between ions), admitted under an HBM budget that
  holds three at a time, each added as another finishes; per run, the same
  comparison with the oracle and what FP32 accumulation of the run's per-step
  increments (extracted charge, energy to the walls) would have cost over 1e7
  steps against the library's 64-bit accumulators.

`python -m pytest tests/test_gpu_scans.py -m gpu -s` prints both tables.
"""
import dataclasses

import numpy as np
import pytest

from oracle import oracle as O
from paper_1507_03392_gb300 import inputs as I

pytestmark = pytest.mark.gpu
QE = 1.602176634e-19


@pytest.fixture(scope="module")
def E():
    from paper_1507_03392_gb300 import ecris
    return ecris


def bound(g, o):
    g, o = np.asarray(g, np.float64), np.asarray(o, np.float64)
    return np.maximum(0.01 * o, 3.0 * np.sqrt(g + o))


def worst(g, o):
    """largest |g - o| / bound over the charge states"""
    g, o = np.asarray(g, np.float64), np.asarray(o, np.float64)
    return float((np.abs(g - o) / np.maximum(bound(g, o), 1e-300)).max())


def fp32_long(xs, total_steps=10_000_000):
    """relative error of summing a run's per-step increments in FP32 over
    total_steps steps (the increments repeated), against the exact sum"""
    xs = np.asarray(xs, dtype=np.float64)
    reps = max(1, total_steps // max(1, len(xs)))
    tiled = np.tile(xs, reps)
    exact = tiled.sum(dtype=np.float64)
    acc = np.cumsum(tiled.astype(np.float32), dtype=np.float32)[-1]
    return abs(float(acc) - exact) / abs(exact) if exact else 0.0


def test_gas_flow_scan_per_run_currents(E, capsys):
    idx = [0, 9, 18, 27, 36, 45, 54, 63]
    steps = 2000
    wls = []
    for i in idx:
        wl = I.config_oxygen_scan(i, n=20_000)
        wl.params = dataclasses.replace(wl.params, dt=1e-7)
        wls.append(wl)
    states = [I.make_particles(wl) for wl in wls]
    nes = [I.make_ne_cells(wl) for wl in wls]
    b = E.Batch()
    hs = [b.add(wl.params, st, ne_cells=ne) for wl, st, ne in zip(wls, states, nes)]
    tune = b.autotune(trial_steps=2)   # the trials are undone
    b.step(steps)
    diags = [b.diag(h) for h in hs]
    b.close()
    rows, bad = [], []
    for i, wl, st, ne, d in zip(idx, wls, states, nes, diags):
        rp = wl.params
        qs = rp.species.qmax + 1
        orc = O.OracleRun(rp, st, ne_cells=ne, deposit=False)
        orc.step(steps)
        ext_g, ext_o = d["extracted"][:qs].astype(np.int64), orc.extracted()[:qs]
        alive_g = d["alive_by_q"][:qs].astype(np.int64)
        alive_o = np.bincount(orc.q, minlength=qs)[:qs]
        charges = np.arange(qs, dtype=np.float64)
        cur_g, cur_o = float((charges * ext_g).sum()), float((charges * ext_o).sum())
        cur_b = max(0.01 * cur_o, 3.0 * np.sqrt((charges ** 2 * (ext_g + ext_o)).sum()))
        rows.append((i, rp.n0_cm3, int(ext_g.sum()), int(ext_o.sum()), cur_g, cur_o, worst(ext_g, ext_o),
                     worst(alive_g, alive_o)))
        if worst(ext_g, ext_o) > 1.0 or worst(alive_g, alive_o) > 1.0 or abs(cur_g - cur_o) > cur_b:
            bad.append((i, ext_g, ext_o, alive_g, alive_o))
    with capsys.disabled():
        print(f"\n[gas-flow scan, 8 of 64 runs in one batch, tuned {tune}, O 2e4 each, dt 1e-7 s, {steps} steps]")
        print("  run   n0 (cm^-3)  extracted GPU / oracle   charge current GPU / oracle (e per run)  "
              "worst |dev|/bound: extracted, in chamber")
        for i, n0, eg, eo, cg, co, we, wa in rows:
            print(f"  {i:3d}  {n0:9.2e}   {eg:7d} / {eo:<7d}       {cg:9.0f} / {co:<9.0f}"
                  f"                       {we:5.2f}, {wa:5.2f}")
    assert not bad, bad


def test_power_scan_per_run_accumulation(E, capsys):
    idx = [0, 21, 42, 63, 84, 105]
    steps = 1500
    wls = []
    for i in idx:
        wl = I.config_power_scan(i, n=20_000)
        wl.params = dataclasses.replace(wl.params, dt=1e-7)
        wls.append(wl)
    states = [I.make_particles(wl) for wl in wls]
    nes = [I.make_ne_cells(wl) for wl in wls]
    rp0 = wls[0].params
    need = E.ecris_run_bytes(20_000, rp0.nx, rp0.ny, rp0.nz, 1)
    b = E.Batch(hbm_budget=int(3.5 * need))
    queue = list(range(len(wls)))
    active = {}                        # handle -> run index
    done_steps = {}
    incr = {k: ([], []) for k in range(len(wls))}
    last = {}
    final = {}
    peak_active = 0
    while queue or active:
        while queue:                    # admit while the budget allows
            k = queue[0]
            try:
                h = b.add(wls[k].params, states[k], ne_cells=nes[k])
            except E.EcrisError as ex:
                assert ex.status == E.ECRIS_ENOMEM
                break
            queue.pop(0)
            active[h] = k
            done_steps[h] = 0
            last[h] = (0.0, 0.0)
        peak_active = max(peak_active, len(active))
        b.step(1)
        for h in list(active):
            k = active[h]
            d = b.diag(h)
            qs = wls[k].params.species.qmax + 1
            qsum = float((np.arange(qs) * d["extracted"][:qs]).sum())
            incr[k][0].append(qsum - last[h][0])
            incr[k][1].append(d["ke_lost_eV"] - last[h][1])
            last[h] = (qsum, d["ke_lost_eV"])
            done_steps[h] += 1
            if done_steps[h] == steps:
                final[k] = d
                b.remove(h)
                del active[h]
    b.close()
    assert peak_active == 3 and len(final) == len(wls)
    rows, bad = [], []
    for k, (i, wl, st, ne) in enumerate(zip(idx, wls, states, nes)):
        rp = wl.params
        qs = rp.species.qmax + 1
        d = final[k]
        orc = O.OracleRun(rp, st, ne_cells=ne, deposit=False)
        orc.step(steps)
        ext_g, ext_o = d["extracted"][:qs].astype(np.int64), orc.extracted()[:qs]
        alive_g = d["alive_by_q"][:qs].astype(np.int64)
        alive_o = np.bincount(orc.q, minlength=qs)[:qs]
        ke_g, ke_o = d["ke_lost_eV"], orc.tally.ke_lost_eV
        q32 = fp32_long(incr[k][0])
        ke32 = fp32_long(incr[k][1])
        rows.append((i, rp.ne_in_cm3, rp.Te_warm_eV, worst(ext_g, ext_o), worst(alive_g, alive_o),
                     abs(ke_g - ke_o) / max(ke_o, 1e-300), q32, ke32, int(ext_g.sum()), int(ext_o.sum())))
        if worst(ext_g, ext_o) > 1.0 or worst(alive_g, alive_o) > 1.0:
            bad.append((i, ext_g, ext_o, alive_g, alive_o))
    with capsys.disabled():
        print(f"\n[power scan, 6 of 128 runs through one batch under an HBM budget of 3 runs, Ar 2e4 each, "
              f"every process, dt 1e-7 s, {steps} steps each]")
        print("  run  n_e (cm^-3)  T_ew (eV)  worst |dev|/bound: extracted, in chamber | wall energy vs FP64 | "
              "FP32 accumulation over 1e7 steps: extracted charge, wall energy | extracted GPU / oracle")
        for i, ne_, te, we, wa, ker, q32, ke32, eg, eo in rows:
            print(f"  {i:3d}  {ne_:9.2e}  {te:8.0f}   {we:5.2f}, {wa:5.2f}                          | "
                  f"{ker:9.2e}           | {q32:9.2e}, {ke32:9.2e}                                | {eg} / {eo}")
        print("  (the library accumulates extracted counts in 64-bit integers and the wall energy in 64-bit "
              "fixed point, 1 micro-eV a unit: exact sums of its FP32 increments)")
    assert not bad, bad
