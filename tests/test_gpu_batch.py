"""GPU tests of the batched form: many runs advanced by one persistent step
kernel over a shared work list, replayed as a CUDA graph.  Every run must give
exactly (bit for bit) what it gives alone, whatever else is in the batch, when
runs join and leave, and whatever launch shape the autotuner picks."""
import numpy as np
import pytest

from paper_1507_03392_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def E():
    from paper_1507_03392_gb300 import ecris
    return ecris


def run_specs():
    specs = []
    # argon with every process including Coulomb collisions
    rp = I.RunParams(nx=16, ny=16, nz=32, ne_in_cm3=2e12, ne_out_cm3=2e11, n0_cm3=1e11, dt=2e-8,
                     flags=I.F_ALL, seed=31)
    wl = I.Workload("a", rp, n=3001, steps=0, atom_fraction=0.5, ion_qmax_init=8, ion_T_eV=10.0,
                    atoms_fill_chamber=True, zone_box=(0.012, 0.15, 0.22))
    specs.append((rp, I.make_particles(wl, seed=31), I.make_efield(rp, 2e3, -1e3)))
    # oxygen, no collisions between ions, another mesh and time step
    rp = I.RunParams(species=I.OXYGEN, nx=8, ny=8, nz=16, ne_in_cm3=5e11, n0_cm3=3e11, dt=5e-9,
                     flags=I.F_ALL_NO_COULOMB, seed=32)
    wl = I.Workload("o", rp, n=5000, steps=0, atom_fraction=0.75, ion_qmax_init=6, ion_T_eV=5.0,
                    atoms_fill_chamber=True)
    specs.append((rp, I.make_particles(wl, seed=32), None))
    # the small argon run (atoms only at the start)
    wl = I.config_small(n=2500, steps=0)
    specs.append((wl.params, I.make_particles(wl), None))
    return specs


def alone(E, rp, st, Ef, steps):
    run = E.Run(rp, E=Ef)
    run.load(st)
    run.step(steps)
    out = (run.state(), run.diag(grids=True))
    run.close()
    return out


def same(a, b):
    ga, da = a
    gb, db = b
    for k in ("x", "y", "z", "vx", "vy", "vz", "meta"):
        assert np.array_equal(ga[k], gb[k]), k
    for k in ("extracted", "lost", "alive_by_q", "cell_count", "cell_charge"):
        assert np.array_equal(da[k], db[k]), k
    assert da["ke_lost_eV"] == db["ke_lost_eV"]
    assert da["coulomb_collisions"] == db["coulomb_collisions"]
    assert da["steps"] == db["steps"]


def test_each_run_in_a_batch_equals_the_run_alone(E):
    specs = run_specs()
    steps = 20
    ref = [alone(E, rp, st, Ef, steps) for rp, st, Ef in specs]
    b = E.Batch()
    hs = [b.add(rp, st, E=Ef) for rp, st, Ef in specs]
    b.step(steps)
    for h, r in zip(hs, ref):
        same((b.state(h), b.diag(h, grids=True)), r)
    b.close()


def test_runs_join_and_leave(E):
    specs = run_specs()
    (rpa, sta, Efa), (rpb, stb, Efb), (rpc, stc, Efc) = specs
    b = E.Batch()
    ha = b.add(rpa, sta, E=Efa)
    hb = b.add(rpb, stb, E=Efb)
    b.step(7)
    b.remove(ha)
    hc = b.add(rpc, stc, E=Efc)
    b.step(9)
    same((b.state(hb), b.diag(hb, grids=True)), alone(E, rpb, stb, Efb, 16))
    same((b.state(hc), b.diag(hc, grids=True)), alone(E, rpc, stc, Efc, 9))
    b.close()


def test_memory_budget_admission(E):
    specs = run_specs()
    rp, st, Ef = specs[1]
    need = E.ecris_run_bytes(len(st["x"]), rp.nx, rp.ny, rp.nz, 0)
    b = E.Batch(hbm_budget=int(2.5 * need))
    b.add(rp, st)
    h2 = b.add(rp, st)
    with pytest.raises(E.EcrisError) as ei:
        b.add(rp, st)
    assert ei.value.status == E.ECRIS_ENOMEM and "budget" in str(ei.value)
    used, budget = b.memory()
    assert used == 2 * need and budget == int(2.5 * need)
    b.remove(h2)
    b.add(rp, st)          # room again
    b.close()


def test_autotune_keeps_results_and_time(E):
    # the tuner's trial steps are undone: after it the runs stand where they
    # stood, and stepping on gives what the runs give alone
    specs = run_specs()
    b = E.Batch()
    hs = [b.add(rp, st, E=Ef) for rp, st, Ef in specs]
    b.step(3)
    before = [(b.state(h), b.diag(h, grids=True)) for h in hs]
    t = b.autotune(trial_steps=2)
    assert t["sort_every"] in (8, 32, 128, 256, 512) and t["blocks_per_sm"] >= 1
    shapes = [(a, v, 2) for a in (128, 256, 512) for v in (1, 2, 4)] + [(128, 2, 3), (256, 1, 3), (256, 2, 3)]
    assert (t["threads"], t["particles_per_thread"], t["stages"]) in shapes
    for h, ref in zip(hs, before):
        same((b.state(h), b.diag(h, grids=True)), ref)
    b.step(5)
    for h, (rp, st, Ef) in zip(hs, specs):
        same((b.state(h), b.diag(h, grids=True)), alone(E, rp, st, Ef, 8))
    b.close()


@pytest.mark.parametrize("threads", [128, 256, 512])
def test_every_launch_shape_gives_the_same_results(E, threads):
    # threads per block x particles per thread x pipeline stages change the
    # tiles a block streams and the work list; each run's result is that of
    # the run alone
    specs = run_specs()
    refs = [alone(E, rp, st, Ef, 7) for rp, st, Ef in specs]
    shapes = [(v, 2) for v in (1, 2, 4)] + {128: [(2, 3)], 256: [(1, 3), (2, 3)], 512: []}[threads]
    for vec, stages in shapes:
        b = E.Batch()
        b.set_tuning(sort_every=4, threads=threads, particles_per_thread=vec, stages=stages)
        hs = [b.add(rp, st, E=Ef) for rp, st, Ef in specs]
        b.step(7)
        for h, ref in zip(hs, refs):
            same((b.state(h), b.diag(h, grids=True)), ref)
        b.close()


def test_set_tuning_rejects_unknown_shapes(E):
    b = E.Batch()
    with pytest.raises(E.EcrisError):
        b.set_tuning(threads=384, particles_per_thread=2)
    with pytest.raises(E.EcrisError):
        b.set_tuning(threads=512, particles_per_thread=2, stages=3)
    with pytest.raises(E.EcrisError):
        b.set_tuning(sort_every=0)
    b.close()


def test_profiled_steps_keep_results(E):
    """With timing on, the batch launches its kernels one by one instead of
    replaying the graph; results must not change."""
    specs = run_specs()
    b = E.Batch()
    hs = [b.add(rp, st, E=Ef) for rp, st, Ef in specs]
    b.step(3)
    b.set_profiling(True)
    b.step(4)
    p = b.profile()
    b.set_profiling(False)
    b.step(2)
    assert p["step_launches"] == 4 and p["step_ms"] > 0
    assert p["coulomb_launches"] > 0 and p["coulomb_launches"] % 4 == 0   # one run has collisions: the same kernels each step
    for h, (rp, st, Ef) in zip(hs, specs):
        same((b.state(h), b.diag(h, grids=True)), alone(E, rp, st, Ef, 9))
    b.close()
