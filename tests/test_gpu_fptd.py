"""GPU parity of the first-passage time distribution (Sec. III.D), through
the C ABI: the closed-form flights of the oracle pins, the distribution of a
busy run against the oracle in lock-step, and a batch run against the same
run alone."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1507_03392_gb300 import inputs as I
from tests import parity as P
from tests import test_oracle_fptd as T

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def E():
    from paper_1507_03392_gb300 import ecris
    return ecris


def _f32(st):
    out = {k: np.asarray(v, np.float32) for k, v in st.items() if k != "q"}
    out["q"] = np.asarray(st["q"]).astype(np.uint8)
    return out


def test_flight_times_closed_form(E):
    rp = I.RunParams(species=T.AR1, B_ecr=100.0, ne_in_cm3=1e20, nx=8, ny=8, nz=32, dt=1e-9,
                     flags=I.F_PUSH | I.F_IONIZE | I.F_RECYCLE)
    d = 1e5 * rp.dt
    ages = [1, 2, 3, 4, 5, 7, 9, 16, 17, 100, 333, 1000, 1500]
    z0 = [rp.L - (a + 0.5) * d for a in ages]
    st = T._axis_run(rp, z0 + z0, [1e5] * (2 * len(ages)), [0] * len(ages) + [1] * len(ages))
    run = E.Run(rp)
    run.load(_f32(st))
    run.step(max(ages) + 2)
    f = run.fptd()
    want = np.zeros((2, E.FPTD_BINS), dtype=np.uint64)
    for a in ages:
        want[1, O.fptd_bin(a)] += 1
    assert np.array_equal(f["hist"], want)
    assert int(f["age_sum"][1]) == sum(ages) and int(f["age_sum"][0]) == 0
    assert run.diag()["extracted"][1] == 2 * len(ages)
    # a new load clears the clock and the distribution
    run.load(_f32(st))
    assert run.fptd()["hist"].sum() == 0
    run.close()


def test_late_birth_closed_form(E):
    rp = I.RunParams(species=T.AR1, B_ecr=100.0, nx=8, ny=8, nz=32, dt=1e-9,
                     flags=I.F_PUSH | I.F_IONIZE | I.F_RECYCLE)
    ne = np.zeros(rp.ncells, dtype=np.float32)
    ne[rp.ncells // 2:] = 1e20
    K = 400
    d = (rp.L / 2) / K
    late = [1, 5, 30, 200]
    z0 = [rp.L / 2 - (b + 0.5) * d for b in late]
    st = T._axis_run(rp, z0, [d / rp.dt] * len(late), [0] * len(late))
    run = E.Run(rp, ne_cells=ne)
    run.load(_f32(st))
    run.step(K + max(late) + 2)
    f = run.fptd()
    assert int(f["hist"][1, O.fptd_bin(K)]) == len(late) and int(f["hist"].sum()) == len(late)
    assert int(f["age_sum"][1]) == K * len(late)
    run.close()


def aperture_case(seed, flags, n=6001, k=2000):
    """A busy all-warm chamber (every process on) with k fast atoms just in
    front of the aperture, so that ions created from them are extracted
    within tens of steps."""
    rp = I.RunParams(nx=16, ny=16, nz=32, B_ecr=100.0, ne_in_cm3=3e12, n0_cm3=3e11, dt=3e-8,
                     Te_warm_eV=500.0, flags=flags, seed=seed)
    wl = I.Workload("fptd", rp, n=n, steps=0, atom_fraction=0.6, ion_qmax_init=4, ion_T_eV=200.0,
                    atoms_fill_chamber=True, zone_box=(0.02, 0.05, 0.29))
    st = I.make_particles(wl, seed=seed)
    rng = np.random.default_rng(seed)
    idx = np.nonzero(np.asarray(st["q"]) == 0)[0][:k]
    r = 0.9 * rp.r_ap * np.sqrt(rng.random(len(idx)))
    ph = 2 * np.pi * rng.random(len(idx))
    st["x"][idx] = r * np.cos(ph)
    st["y"][idx] = r * np.sin(ph)
    st["z"][idx] = rp.L - 0.02 * rng.random(len(idx))
    st["vz"][idx] = rng.uniform(1e4, 5e4, len(idx))
    st["vx"][idx] = rng.normal(0, 300, len(idx))
    st["vy"][idx] = rng.normal(0, 300, len(idx))
    return rp, st


def test_busy_run_matches_oracle(E):
    # the histogram of both sides, up to the particles whose outcome was guarded
    rp, st = aperture_case(21, I.F_ALL_NO_COULOMB)
    run = E.Run(rp)
    run.load(st)
    t, orc = P.lockstep(run, rp, st, 150)
    assert t["q"] == 0 and t["events"] == 0 and t["pos"] == 0 and t["vel"] == 0, t["first_bad"]
    f = run.fptd()
    q1 = rp.species.qmax + 1
    assert orc.fptd_hist.sum() >= 100, orc.fptd_hist.sum()
    diff = np.abs(f["hist"].astype(np.int64) - orc.fptd_hist[:q1]).sum()
    assert diff <= 2 * t["accepted"], (diff, t["accepted"])
    if diff == 0:
        assert np.array_equal(f["age_sum"].astype(np.int64), orc.fptd_sum[:q1])
    run.close()


def test_batch_equals_run_alone(E):
    rp, st = aperture_case(22, I.F_ALL, n=8001)
    run = E.Run(rp)
    run.load(st)
    run.step(200)
    b = E.Batch()
    h = b.add(rp, st)
    b.step(200)
    fa, fb = run.fptd(), b.fptd(h)
    assert fa["hist"].sum() >= 100
    assert np.array_equal(fa["hist"], fb["hist"]) and np.array_equal(fa["age_sum"], fb["age_sum"])
    b.close()
    run.close()
