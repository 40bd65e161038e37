"""Pins of the oracle's first-passage time distribution (Sec. III.D): the age
of an extracted ion counts the steps since its creation by ionisation of an
atom.

The closed forms use ions on the chamber axis moving along z: there B is
along the axis, so the push leaves v unchanged and the extraction step
follows from the kinematics alone.  A one-charge-state species keeps a
created ion at Q = 1."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1507_03392_gb300 import inputs as I

AR1 = I.Species("Ar1", 40.0, 18, 1)


def _lower_edge(b):
    e, m = divmod(b, 4)
    return (1 << e) * (4 + m) // 4


def test_bin_edges_by_brute_force():
    # bin 4e + m holds the ages [2^e (1 + m/4), 2^e (1 + (m + 1)/4)) for e >= 2;
    # below 4 every age has its own bin (0, 4, 6, 8)
    prev = -1
    for a in range(1, 20000):
        b = O.fptd_bin(a)
        assert b >= prev
        prev = b
        if a >= 4:
            assert _lower_edge(b) <= a < _lower_edge(b + 1)
    assert [O.fptd_bin(a) for a in (1, 2, 3)] == [0, 4, 6]
    assert O.fptd_bin(2 ** 30 - 1) == O.FPTD_BINS - 1


def _axis_run(rp, z0, vz, q):
    n = len(z0)
    st = {k: np.zeros(n) for k in ("x", "y", "vx", "vy")}
    st["z"] = np.asarray(z0, dtype=np.float64)
    st["vz"] = np.asarray(vz, dtype=np.float64)
    st["q"] = np.asarray(q, dtype=np.int32)
    return st


def test_atoms_ionised_at_once_give_their_flight_times():
    # every cell warm with an n_e so high that an atom ionises in its first
    # step (p = 1): born at step 0, extracted in the step where it passes L
    rp = I.RunParams(species=AR1, B_ecr=100.0, ne_in_cm3=1e20, nx=8, ny=8, nz=32, dt=1e-9,
                     flags=I.F_PUSH | I.F_IONIZE | I.F_RECYCLE)
    d = 1e5 * rp.dt                                  # 0.1 mm per step
    ages = [1, 2, 3, 4, 5, 7, 9, 16, 17, 100, 333, 1000, 1500]
    z0 = [rp.L - (a + 0.5) * d for a in ages]
    # the same flights for ions loaded as ions: their birth is unknown
    st = _axis_run(rp, z0 + z0, [1e5] * (2 * len(ages)), [0] * len(ages) + [1] * len(ages))
    r = O.OracleRun(rp, st)
    r.step(1)
    assert np.all((r.events[: len(ages)] & O.EV_IONIZE) != 0)
    r.step(max(ages) + 1)
    want = np.zeros_like(r.fptd_hist)
    for a in ages:
        want[1, O.fptd_bin(a)] += 1
    assert np.array_equal(r.fptd_hist, want)
    assert r.fptd_sum[1] == sum(ages) and r.fptd_sum[0] == 0
    # all of them were extracted
    assert r.extracted()[1] == 2 * len(ages)


def test_birth_is_the_ionisation_step():
    # no electrons below the mid-plane: an atom ionises in the step that takes
    # it past z = L/2 and is extracted K steps later
    rp = I.RunParams(species=AR1, B_ecr=100.0, nx=8, ny=8, nz=32, dt=1e-9,
                     flags=I.F_PUSH | I.F_IONIZE | I.F_RECYCLE)
    ne = np.zeros(rp.ncells, dtype=np.float32)
    ne[rp.ncells // 2:] = 1e20
    K = 400
    d = (rp.L / 2) / K
    late = [1, 5, 30, 200]
    z0 = [rp.L / 2 - (b + 0.5) * d for b in late]
    st = _axis_run(rp, z0, [d / rp.dt] * len(late), [0] * len(late))
    r = O.OracleRun(rp, st, ne_cells=ne)
    r.step(K + max(late) + 2)
    assert r.fptd_hist[1, O.fptd_bin(K)] == len(late)
    # the summed ages pin them exactly (ages counted from the load would sum
    # to K * 4 + 236 here)
    assert r.fptd_hist.sum() == len(late) and r.fptd_sum[1] == K * len(late)

