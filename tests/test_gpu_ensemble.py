"""Ensemble parity of the FP32 CUDA path with the FP64 oracle (GPU): the
charge-state distribution and the extracted currents by charge state (Sec. II:
the model's output is the charge-state distribution of the extracted ions;
Sec. III: the currents).

The GPU and the oracle each run freely from the same initial state with the
same counter-based random words.  Their histories stay identical until a
decision within rounding of its surface goes the other way; after that a
particle's history, and through it the ensemble, evolves independently.  With
collisions between ions a single flip re-pairs a cell and the two runs soon
become independent samples of the same process, so a count's difference has
the variance of a difference of two Poisson counts, N_gpu + N_oracle.  The
bar: every charge state's count within max(1 % of the oracle's,
3 sqrt(N_gpu + N_oracle)).  The extraction-heavy run below (no collisions
between ions, histories shared but for the flips) reaches N >= 1e5 in its
leading charge states, and there the test asserts the 1 % bar on its own.  The
runs of the two batched scans extract few ions in any affordable number of
steps (a 1 cm aperture in a 6.4 cm chamber, a mirror), so their bins are held
to the 3 sigma bound and their event counts are printed beside the result.
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


def extraction_heavy():
    """Synthetic stand-in built to extract many ions: a nearly flat 1 T
    solenoid (no mirror to reflect ions from the extraction plate, no
    hexapole), the ECR threshold raised to 1.5 T so the whole chamber holds
    warm electrons (n_e 3e13 cm^-3, 1 keV), a 3 cm aperture, 2 eV re-emitted
    gas so the neutrals spread fast, dt 0.1 us."""
    rp = I.RunParams(species=I.OXYGEN, nx=16, ny=16, nz=32, r_ap=0.030, B_inj=1.05, B_min=1.0, B_ext=1.02,
                     B_hex=0.0, B_ecr=1.5, ne_in_cm3=3e13, ne_out_cm3=3e12, Te_warm_eV=1000.0, n0_cm3=1e11,
                     T0_eV=2.0, dt=1e-7, flags=I.F_ALL_NO_COULOMB, seed=4242)
    wl = I.Workload("o_extraction_heavy", rp, n=20_000, steps=15_000, atom_fraction=0.5, ion_qmax_init=3,
                    ion_T_eV=1.0, atoms_fill_chamber=True, zone_box=(0.02, 0.02, 0.28))
    return wl


def cases():
    out = [("O 2e4, extraction-heavy stand-in (flat 1 T, 3 cm aperture), dt 1e-7 s, 15000 steps",
            extraction_heavy(), 15_000)]
    wl = I.config_oxygen_scan(63, n=20_000)
    wl.params = dataclasses.replace(wl.params, dt=1e-7)
    out.append((f"gas-flow scan run 63 (O, n0 {wl.params.n0_cm3:.1e} cm^-3, no ion-ion), 2e4, dt 1e-7 s, "
                "6000 steps", wl, 6000))
    wl = I.config_power_scan(5, n=20_000)
    wl.params = dataclasses.replace(wl.params, dt=1e-7)
    p = wl.params
    out.append((f"power scan run 5 (Ar, n_e {p.ne_in_cm3:.1e} cm^-3, T_ew {p.Te_warm_eV:.0f} eV, every process "
                "with ion-ion), 2e4, dt 1e-7 s, 3000 steps", wl, 3000))
    return out


def bound(g, o):
    """max(1 % of the oracle's count, 3 sigma of the difference of two
    independent Poisson counts)"""
    g, o = np.asarray(g, np.float64), np.asarray(o, np.float64)
    return np.maximum(0.01 * o, 3.0 * np.sqrt(g + o))


def within(g, o):
    return np.abs(np.asarray(g, np.float64) - np.asarray(o, np.float64)) <= bound(g, o)


@pytest.mark.parametrize("k", range(3))
def test_ensemble_csd_and_currents(E, k, capsys):
    name, wl, steps = cases()[k]
    rp = wl.params
    st = I.make_particles(wl)
    ne = I.make_ne_cells(wl)
    run = E.Run(rp, ne_cells=ne)
    run.load(st)
    run.step(steps)
    d = run.diag()
    run.close()
    orc = O.OracleRun(rp, st, ne_cells=ne, deposit=False)
    orc.step(steps)
    qs = rp.species.qmax + 1
    ext_g, ext_o = d["extracted"][:qs].astype(np.int64), orc.extracted()[:qs]
    alive_g = d["alive_by_q"][:qs].astype(np.int64)
    alive_o = np.bincount(orc.q, minlength=qs)[:qs]
    charges = np.arange(qs, dtype=np.float64)
    cur_g, cur_o = float((charges * ext_g).sum()), float((charges * ext_o).sum())
    with capsys.disabled():
        print(f"\n[{name}]")
        print("   Q   extracted GPU / oracle      rel     bound | in chamber GPU / oracle      rel")
        for q in range(qs):
            if ext_o[q] or ext_g[q] or alive_o[q] or alive_g[q]:
                re = abs(ext_g[q] - ext_o[q]) / max(ext_o[q], 1)
                ra = abs(alive_g[q] - alive_o[q]) / max(alive_o[q], 1)
                bq = float(bound(ext_g[q], ext_o[q])) / max(ext_o[q], 1)
                print(f"  {q:2d} {ext_g[q]:10d} / {ext_o[q]:<10d} {re:8.2e} {bq:8.2e} | "
                      f"{alive_g[q]:8d} / {alive_o[q]:<8d} {ra:8.2e}")
        print(f"  extracted charge (sum Q N): GPU {cur_g:.0f}, oracle {cur_o:.0f}, rel "
              f"{abs(cur_g - cur_o) / max(cur_o, 1):.2e}; charge states with >= 1e5 events: "
              f"{int((ext_o >= 100_000).sum())}")
    assert within(ext_g, ext_o).all(), (ext_g, ext_o)
    assert within(alive_g, alive_o).all(), (alive_g, alive_o)
    assert abs(cur_g - cur_o) <= max(0.01 * cur_o, 3.0 * np.sqrt((charges ** 2 * (ext_g + ext_o)).sum()))
    if k == 0:
        # the 1 % bar is exercised: at least two charge states carry >= 1e5
        # extraction events (Poisson error below 0.32 %)
        assert (ext_o >= 100_000).sum() >= 2, ext_o
        big = ext_o >= 100_000
        assert (np.abs(ext_g[big] - ext_o[big]) <= 0.01 * ext_o[big]).all()
    else:
        assert ext_o.sum() >= 100, ext_o
