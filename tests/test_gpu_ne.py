"""GPU parity of the self-consistent electron density (Sec. II: n_e equals the
ion charge density, by charge neutrality), through the C ABI.

* Resting ions: the device's n_e equals the closed form w sum(Q) / V_cell of
  the placement, its delta equals the oracle's, and the time average restarts
  at each update.
* Lock-step with updates every 20 steps: the cell records of both sides agree
  wherever their deposits agree, and the particles stay in parity across the
  updates (the MCC block then reads the new n_e and delta).
* A run in a batch updated at the same steps as the run alone gives the same
  records and the same results, bit for bit.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1507_03392_gb300 import inputs as I
from tests import parity as P
from tests import test_oracle_ne as T

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def E():
    from paper_1507_03392_gb300 import ecris
    return ecris


def _delta_close(got, want):
    floor = 1e-6 * max(1e-30, float(np.abs(want).max()))
    return np.abs(got.astype(np.float64) - want) <= 1e-5 * np.abs(want) + floor


def test_resting_ions_closed_form(E):
    rp = I.RunParams(nx=8, ny=8, nz=16, flags=0, weight=3e7)
    rng = np.random.default_rng(12)
    cq = []
    for _ in range(3001):
        while True:
            ix, iy = rng.integers(1, rp.nx - 1, size=2)
            cx, cy, _ = T._centre(rp, ix, iy, 0)
            if cx * cx + cy * cy < (0.8 * rp.R0) ** 2:
                break
        cq.append(((int(ix), int(iy), int(rng.integers(0, rp.nz))), int(rng.integers(0, 19))))
    st = T._resting(rp, cq)
    st32 = {k: np.asarray(v, np.float32) for k, v in st.items() if k != "q"}
    st32["q"] = st["q"].astype(np.uint8)
    want = np.zeros(rp.ncells)
    for (ix, iy, iz), q in cq:
        want[T._cell_index(rp, ix, iy, iz)] += q
    want *= rp.weight / T._volume(rp)

    run = E.Run(rp)
    run.load(st32)
    with pytest.raises(E.EcrisError) as ei:
        run.update_ne()                      # no step yet
    assert ei.value.status == E.ECRIS_ESTATE
    before = run.cells()
    assert before["ne"].max() > 0            # the prescribed n_e
    run.step(7)
    run.update_ne()
    c = run.cells()
    # FP64 from the integer deposit, rounded once to FP32
    assert np.allclose(c["ne"], want, rtol=1.2e-7, atol=0)
    assert np.all(c["ne"][want == 0] == 0)
    orc = O.OracleRun(rp, st)
    orc.step(7)
    orc.update_ne()
    assert np.all(_delta_close(c["delta_x"], orc.dlx)) and np.all(_delta_close(c["delta_y"], orc.dly))
    assert np.all(c["delta_x"][want == 0] == 0) and np.all(c["delta_y"][want == 0] == 0)
    # the average restarts at the update: the same density from the next 3 steps
    run.step(3)
    run.update_ne()
    assert np.allclose(run.cells()["ne"], want, rtol=1.2e-7, atol=0)
    run.close()


def _cells_of(rp, x, y, z):
    dx, dy, dz = 2 * rp.R0 / rp.nx, 2 * rp.R0 / rp.ny, rp.L / rp.nz
    ix = np.clip(np.floor((np.asarray(x, np.float64) + rp.R0) / dx).astype(np.int64), 0, rp.nx - 1)
    iy = np.clip(np.floor((np.asarray(y, np.float64) + rp.R0) / dy).astype(np.int64), 0, rp.ny - 1)
    iz = np.clip(np.floor(np.asarray(z, np.float64) / dz).astype(np.int64), 0, rp.nz - 1)
    return (iz * rp.ny + iy) * rp.nx + ix


def _lockstep_ne(E, update_every, steps=100):
    rp = I.RunParams(nx=16, ny=16, nz=32, ne_in_cm3=3e12, ne_out_cm3=3e11, n0_cm3=3e11, dt=3e-8,
                     Te_warm_eV=500.0, flags=I.F_ALL_NO_COULOMB, seed=9, weight=2e9)
    wl = I.Workload("ne", rp, n=4001, steps=0, atom_fraction=0.3, ion_qmax_init=8, ion_T_eV=60.0,
                    atoms_fill_chamber=True, zone_box=(0.02, 0.05, 0.29))
    st = I.make_particles(wl, seed=9)
    Ef = I.make_efield(rp, 4e3, -2e3)
    run = E.Run(rp, E=Ef)
    run.load(st)
    orc = O.OracleRun(rp, st, E=Ef)
    excused = np.zeros(rp.ncells, dtype=bool)
    out = {"updates": 0, "ions_seen": 0, "excused_particles": 0, "handover": 0, "bad": []}
    for s in range(steps):
        if update_every and s and s % update_every == 0:
            run.update_ne()
            orc.update_ne()
            out["updates"] += 1
            c = run.cells()
            dep = run.diag(grids=True)["cell_charge"].astype(np.int64)
            dq = dep != orc.dep_charge
            ne_bad = np.abs(c["ne"].astype(np.float64) - orc.ne) > 1e-6 * np.abs(orc.ne)
            dl_bad = ~_delta_close(c["delta_x"], orc.dlx) | ~_delta_close(c["delta_y"], orc.dly)
            # records differ only where a guarded particle deposited elsewhere
            # (its cell, and for delta its 3x3 neighbourhood in x-y)
            near = dq.reshape(rp.nz, rp.ny, rp.nx).copy()
            near = near | np.roll(near, 1, 1) | np.roll(near, -1, 1)
            near = near | np.roll(near, 1, 2) | np.roll(near, -1, 2)
            assert not np.any(ne_bad & ~dq) and not np.any(dl_bad & ~near.reshape(-1))
            excused = ne_bad | dl_bad
            assert excused.sum() <= 9 * max(1, int(dq.sum())) and dq.sum() <= 5
            out["ions_seen"] += int((orc.ne > 0).sum())
        g0 = run.state()
        orc.set_state({k: g0[k] for k in P.KEYS + ("q",)})
        orc.status[:] = np.where((g0["meta"] & (1 << 16)) != 0, 1, 0)
        orc.step_index = s
        orc.step(1)
        run.step(1)
        g1 = run.state()
        hit = None
        if excused.any():
            # cells whose electron record the device built from a deposit that
            # differs by a guarded particle: their particles are exempt
            hit = excused[_cells_of(rp, g0["x"], g0["y"], g0["z"])] | \
                excused[_cells_of(rp, orc.x, orc.y, orc.z)]
            out["excused_particles"] += int(hit.sum())
        r = P.compare_step(rp, g1, orc, probes=P.Probes(rp, g0, s, orc), excuse=hit)
        out["handover"] += r["handover"]
        if r["q"] or r["events"] or r["pos"] or r["vel"]:
            i = r["detail"]["i"]
            out["bad"].append({"step": s, **{k: r[k] for k in ("q", "events", "pos", "vel")},
                               "before": [float(g0[k][i]) for k in P.KEYS], **r["detail"],
                               "cell": int(_cells_of(rp, g0["x"][i], g0["y"][i], g0["z"][i])),
                               "ne": float(orc.ne[_cells_of(rp, g0["x"][i], g0["y"][i], g0["z"][i])])})
    run.close()
    return out


@pytest.mark.parametrize("update_every", [0, 20])
def test_lockstep_across_updates(E, update_every):
    out = _lockstep_ne(E, update_every)
    if out["bad"]:
        pytest.fail(f"update_every={update_every}: {len(out['bad'])} mismatching steps, first {out['bad'][:3]}")
    if update_every:
        assert out["updates"] == 4 and out["ions_seen"] > 1000
        assert out["excused_particles"] <= 0.01 * 4001 * 100


def test_batch_update_equals_run_alone(E):
    rp = I.RunParams(nx=16, ny=16, nz=32, ne_in_cm3=2e12, ne_out_cm3=2e11, n0_cm3=1e11, dt=2e-8,
                     flags=I.F_ALL, seed=31, weight=5e8)
    wl = I.Workload("b", rp, n=6001, steps=0, atom_fraction=0.5, ion_qmax_init=8, ion_T_eV=10.0,
                    atoms_fill_chamber=True, zone_box=(0.012, 0.15, 0.22))
    st = I.make_particles(wl, seed=31)
    rp2 = I.RunParams(species=I.OXYGEN, nx=8, ny=8, nz=16, ne_in_cm3=5e11, n0_cm3=3e11, dt=5e-9,
                      flags=I.F_ALL_NO_COULOMB, seed=32)
    wl2 = I.Workload("o", rp2, n=3000, steps=0, atom_fraction=0.75, ion_qmax_init=6, ion_T_eV=5.0,
                     atoms_fill_chamber=True)
    st2 = I.make_particles(wl2, seed=32)

    run = E.Run(rp)
    run.load(st)
    b = E.Batch()
    h = b.add(rp, st)
    h2 = b.add(rp2, st2)
    for k in range(3):
        run.step(16)
        b.step(16)
        run.update_ne()
        b.update_ne(h)
        ca, cb = run.cells(), b.cells(h)
        for key in ("ne", "delta_x", "delta_y"):
            assert np.array_equal(ca[key], cb[key]), (k, key)
    run.step(16)
    b.step(16)
    da, db = run.diag(grids=True), b.diag(h, grids=True)
    for key in ("extracted", "lost", "alive_by_q", "cell_charge"):
        assert np.array_equal(da[key], db[key]), key
    assert da["ke_lost_eV"] == db["ke_lost_eV"]
    # the other run of the batch kept its prescribed n_e and delta
    c2 = b.cells(h2)
    lone = E.Run(rp2)
    c2_lone = lone.cells()
    lone.close()
    for key in ("ne", "delta_x", "delta_y"):
        assert np.array_equal(c2[key], c2_lone[key]), key
    sa, sb = run.state(), b.state(h)
    for key in ("x", "y", "z", "vx", "vy", "vz", "meta"):
        assert np.array_equal(sa[key], sb[key]), key
    b.close()
    run.close()
