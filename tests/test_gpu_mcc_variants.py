"""GPU parity of the opt-in processes and variants (Sec. II collision block;
Secs. III.C, IV) through the C ABI: double ionisation, elastic ion-atom
scattering, recombination, warm reflected atoms and isotropic heating, in
lock-step with the oracle, and a batch run against the same run alone."""
import dataclasses

import numpy as np
import pytest

from oracle import oracle as O
from paper_1507_03392_gb300 import inputs as I
from tests import parity as P
from tests import test_gpu_parity as G
from tests import test_oracle_mcc_variants as V

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def E():
    from paper_1507_03392_gb300 import ecris
    return ecris


def _variant_case(seed=4):
    rp, st, Ef = G.busy_case(seed=seed)
    rp = dataclasses.replace(rp, flags=rp.flags | I.F_DOUBLE | I.F_ELASTIC | I.F_RECOMB, T_refl_eV=0.15, k2_factor=0.5,
                             sigma_el1_cm2=2e-14)
    return rp, st, Ef


def test_lockstep_double_elastic_warm_reflection(E):
    rp, st, Ef = _variant_case()
    run = E.Run(rp, E=Ef)
    run.load(st)
    orc = O.OracleRun(rp, st, E=Ef)
    seen = np.zeros(6, dtype=np.int64)
    doubles = 0
    for s in range(60):
        g0 = run.state()
        orc.set_state({k: g0[k] for k in P.KEYS + ("q",)})
        orc.status[:] = np.where((g0["meta"] & (1 << 16)) != 0, 1, 0)
        orc.step_index = s
        orc.step(1)
        run.step(1)
        g1 = run.state()
        r = P.compare_step(rp, g1, orc, probes=P.Probes(rp, g0, s, orc))
        assert not (r["q"] or r["events"] or r["pos"] or r["vel"]), (s, r)
        for b in range(6):
            seen[b] += int(((orc.events >> b) & 1).sum())
        doubles += int(((g1["q"].astype(np.int64) - g0["q"]) >= 2).sum())
    wall, ext, ion, cx, _, el = seen
    assert wall > 50 and ion > 15 and cx > 5 and el > 50 and doubles > 0, (seen, doubles)
    run.close()


def test_lockstep_recombination(E):
    # ions at rest in cold, dense electrons: recombination competes with
    # ionisation for the same word
    rp = V._uniform_params(flags=I.F_RECOMB | I.F_IONIZE, Te_warm_eV=8.0, Te_cold_eV=8.0, ne_in_cm3=1e14,
                           ne_out_cm3=1e14, dt=3e-5)
    st = V._static(4001, 6, rp)
    st32 = {k: np.asarray(v, np.float32) for k, v in st.items() if k != "q"}
    st32["q"] = st["q"].astype(np.uint8)
    run = E.Run(rp)
    run.load(st32)
    t, orc = P.lockstep(run, rp, st32, 12)
    assert t["q"] == 0 and t["events"] == 0 and t["pos"] == 0 and t["vel"] == 0, t["first_bad"]
    g = run.state()
    assert (g["q"] < 6).sum() > 500 and (g["q"] > 6).sum() > 0
    run.close()


def test_lockstep_triple_ionisation(E):
    # ions at rest in dense warm electrons: single, double and triple
    # ionisation and recombination share one word; the triple steps and the
    # top charge states match the oracle particle by particle
    rp = V._uniform_params(species=I.OXYGEN, flags=I.F_IONIZE | I.F_DOUBLE | I.F_RECOMB, Te_warm_eV=3000.0,
                           Te_cold_eV=3000.0, ne_in_cm3=1e13, ne_out_cm3=1e13, k2_factor=1.0, k3_factor=1.0,
                           dt=5e-7)
    st = V._static(4001, 1, rp)
    st["q"][2000:] = rp.species.qmax - 3        # a triple step from here ends at qmax
    st32 = {k: np.asarray(v, np.float32) for k, v in st.items() if k != "q"}
    st32["q"] = st["q"].astype(np.uint8)
    run = E.Run(rp)
    run.load(st32)
    triples = 0
    orc = O.OracleRun(rp, st32)
    for s in range(12):
        g0 = run.state()
        run.step(1)
        orc.step(1)
        g1 = run.state()
        assert np.array_equal(g1["q"].astype(np.int64), orc.q), s
        triples += int(((g1["q"].astype(np.int64) - g0["q"]) == 3).sum())
    assert triples > 20 and g1["q"].max() == rp.species.qmax
    run.close()


def test_warm_reflection_each_particle(E):
    # ions and atoms driven onto the z = 0 flange come back at T_refl and T0
    rp = V._uniform_params(flags=I.F_PUSH | I.F_RECYCLE, T_refl_eV=0.15, dt=1e-9)
    for q in (3, 0):
        st = V._flange_hits(rp, 4001, q)
        st32 = {k: np.asarray(v, np.float32) for k, v in st.items() if k != "q"}
        st32["q"] = st["q"].astype(np.uint8)
        run = E.Run(rp)
        run.load(st32)
        t, orc = P.lockstep(run, rp, st32, 1)
        assert t["q"] == 0 and t["events"] == 0 and t["vel"] == 0 and t["pos"] == 0, t["first_bad"]
        assert t["events_seen"][0] == 4001
        g = run.state()
        M = rp.species.mass_amu * 1.66053906660e-27
        T = 0.15 if q else rp.T0_eV
        vn2 = (g["vz"].astype(np.float64) ** 2).mean() / (2 * T * 1.602176634e-19 / M)
        assert abs(vn2 - 1) < 5 / np.sqrt(4001)
        run.close()


def test_isotropic_heating_cells_and_lockstep(E):
    rp = I.RunParams(B_ecr=100.0, nx=12, ny=12, nz=6, flags=I.F_ALL_NO_COULOMB | I.F_ISOHEAT, dt=1e-8,
                     n0_cm3=1e11, seed=8)
    iy = (np.arange(rp.ncells) // rp.nx) % rp.ny
    ne = (3e11 + 2e10 * iy).astype(np.float32)
    wl = I.Workload("iso", rp, n=3001, steps=0, atom_fraction=0.3, ion_qmax_init=6, ion_T_eV=20.0,
                    atoms_fill_chamber=True)
    st = I.make_particles(wl, seed=8)
    run = E.Run(rp, ne_cells=ne)
    run.load(st)
    c = run.cells()
    assert np.all(c["delta_x"] == 0) and np.all(c["delta_y"] == 0) and c["ne"].max() > 0
    t, orc = P.lockstep(run, rp, st, 30, ne_cells=ne)
    assert t["q"] == 0 and t["events"] == 0 and t["pos"] == 0 and t["vel"] == 0, t["first_bad"]
    # the update of n_e keeps delta at zero
    run.update_ne()
    c = run.cells()
    assert np.all(c["delta_x"] == 0) and np.all(c["delta_y"] == 0)
    run.close()


def test_batch_with_variants_equals_run_alone(E):
    rp, st, Ef = _variant_case(seed=6)
    rp = dataclasses.replace(rp, flags=rp.flags | I.F_COULOMB | I.F_ISOHEAT)
    run = E.Run(rp, E=Ef)
    run.load(st)
    run.step(40)
    b = E.Batch()
    h = b.add(rp, st, E=Ef)
    b.step(40)
    da, db = run.diag(grids=True), b.diag(h, grids=True)
    for key in ("extracted", "lost", "alive_by_q", "cell_charge"):
        assert np.array_equal(da[key], db[key]), key
    assert da["ke_lost_eV"] == db["ke_lost_eV"]
    sa, sb = run.state(), b.state(h)
    for key in ("x", "y", "z", "vx", "vy", "vz", "meta"):
        assert np.array_equal(sa[key], sb[key]), key
    b.close()
    run.close()


def test_invalid_variant_parameters(E):
    rp = dataclasses.replace(G.busy_case()[0], k2_factor=-1.0)
    with pytest.raises(E.EcrisError):
        E.Run(rp)
    rp = dataclasses.replace(G.busy_case()[0], k3_factor=-0.5)
    with pytest.raises(E.EcrisError):
        E.Run(rp)
    rp = dataclasses.replace(G.busy_case()[0], T_refl_eV=float("nan"))
    with pytest.raises(E.EcrisError):
        E.Run(rp)
    rp = dataclasses.replace(G.busy_case()[0], flags=1 << 10)
    with pytest.raises(E.EcrisError):
        E.Run(rp)
