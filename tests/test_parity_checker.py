"""CPU tests of the lock-step checker (tests/parity.py) itself.

A stand-in for the CUDA run is the FP64 oracle stepping a state whose true
positions lie 0.45 FP32 ulp below the FP32 values it exports (which they still
round to), the way the device's exact fixed-point positions lie within half an
ulp of their FP32 export.  Atoms parked exactly on a cell face (z = float32(0.15), a face of the 16-cell
z mesh; vz = 0, so they stay there) then take the decisions of the cell below
while the oracle, handed the exported positions, uses the cell above.  The
checker must explain every such flip by its probes, also with ion-ion
collisions whose pairings the flips change, and must still report mistakes
planted in the stand-in's output (a velocity, a charge state, two swapped
collision partners).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1507_03392_gb300 import inputs as I
from tests import parity as P

Z_FACE = np.float32(0.15)


class OracleStandIn:
    """state()/step() of a CUDA run, computed by the oracle"""

    def __init__(self, rp, st, ne_cells, plant=None):
        self.rp = rp
        self.orc = O.OracleRun(rp, st, ne_cells=ne_cells, deposit=False)
        self.s = 0
        self.plant = plant
        self._shift()

    def _shift(self):
        # true position: the FP32 value moved 0.45 ulp down in z, which still
        # rounds to it; the face z = 0.15 lies 0.4 ulp below float32(0.15)
        z32 = self.orc.z.astype(np.float32)
        ulp = np.spacing(z32).astype(np.float64)
        self.orc.z = np.ascontiguousarray(z32.astype(np.float64) - 0.45 * ulp)
        for k in ("x", "y", "vx", "vy", "vz"):
            setattr(self.orc, k, np.ascontiguousarray(getattr(self.orc, k).astype(np.float32).astype(np.float64)))

    def state(self):
        o = self.orc
        meta = (o.events.astype(np.uint32) << 8) | (o.status.astype(np.uint32) << 16) | o.q.astype(np.uint32)
        out = {k: getattr(o, k).astype(np.float32) for k in P.KEYS}
        out["q"] = o.q.astype(np.uint8)
        out["meta"] = meta
        return out

    def step(self, n=1):
        for _ in range(n):
            self.orc.step_index = self.s
            self.orc.step(1)
            if self.plant is not None and self.plant[0] == self.s:
                self.plant[1](self.orc)
            self.s += 1
            self._shift()


def face_state(rp, seed, n_face=6000, n_ions=3000):
    rng = np.random.default_rng(seed)
    # atoms on the face, at rest in z, inside r < 1.5 cm
    r = 0.015 * np.sqrt(rng.random(n_face))
    th = rng.random(n_face) * 2 * np.pi
    v = rng.normal(0, 300.0, (3, n_face))
    v[2] = 0.0
    # ions in the cells on both sides of the face, away from it
    ri = 0.015 * np.sqrt(rng.random(n_ions))
    ti = rng.random(n_ions) * 2 * np.pi
    zi = 0.15 + rng.choice([-1, 1], n_ions) * rng.uniform(0.002, 0.015, n_ions)
    vi = rng.normal(0, 2000.0, (3, n_ions))
    qi = rng.integers(1, 6, n_ions)
    f32 = np.float32
    return {"x": np.concatenate([r * np.cos(th), ri * np.cos(ti)]).astype(f32),
            "y": np.concatenate([r * np.sin(th), ri * np.sin(ti)]).astype(f32),
            "z": np.concatenate([np.full(n_face, Z_FACE), zi]).astype(f32),
            "vx": np.concatenate([v[0], vi[0]]).astype(f32), "vy": np.concatenate([v[1], vi[1]]).astype(f32),
            "vz": np.concatenate([v[2], vi[2]]).astype(f32),
            "q": np.concatenate([np.zeros(n_face), qi]).astype(np.uint8)}


def setup(coulomb, seed=5):
    fl = (I.F_ALL if coulomb else I.F_ALL_NO_COULOMB) & ~I.F_CX
    rp = I.RunParams(nx=8, ny=8, nz=16, flags=fl, ne_in_cm3=5e12, ne_out_cm3=5e12, dt=2e-8, weight=2e8,
                     seed=seed)
    rng = np.random.default_rng(seed + 1)
    # electron density differing from cell to cell (cm^-3), so the cells on
    # the two sides of the face ionise with different probabilities
    ne = np.exp(rng.uniform(np.log(2e12), np.log(2e13), rp.ncells)).astype(np.float32)
    rp = I.RunParams(**{**rp.__dict__, "ne_out_cm3": 5e12})
    return rp, face_state(rp, seed), ne


@pytest.mark.parametrize("coulomb", [False, True])
def test_flips_at_a_cell_face_are_explained(coulomb):
    rp, st, ne = setup(coulomb)
    run = OracleStandIn(rp, st, ne)
    t, _ = P.lockstep(run, rp, st, 30, ne_cells=ne, vel_rel=5e-5)
    assert t["q"] == 0 and t["events"] == 0 and t["pos"] == 0 and t["vel"] == 0, (t, t["first_bad"])
    # the stand-in really took the other side: the probes explained flips
    assert t["accepted"] >= 10, t


def test_flips_are_reported_without_probes():
    rp, st, ne = setup(False)
    run = OracleStandIn(rp, st, ne)
    orc = O.OracleRun(rp, st, ne_cells=ne)
    bad = 0
    for s in range(25):
        g0 = run.state()
        orc.set_state({k: g0[k] for k in P.KEYS + ("q",)})
        orc.step_index = s
        orc.step(1)
        run.step(1)
        r = P.compare_step(rp, run.state(), orc, vel_rel=5e-5, probes=None)
        bad += r["q"] + r["events"]
    assert bad >= 10


def _far_ion(orc, rp):
    """an ion of the stand-in far from every face and wall"""
    dz = rp.L / rp.nz
    gz = orc.z / dz
    far = (orc.q >= 1) & (np.abs(gz - np.round(gz)) > 0.2) & (orc.x ** 2 + orc.y ** 2 < 0.01 ** 2)
    return int(np.nonzero(far)[0][0])


@pytest.mark.parametrize("coulomb", [False, True])
def test_planted_velocity_error_is_reported(coulomb):
    rp, st, ne = setup(coulomb)

    def plant(o):
        i = _far_ion(o, rp)
        o.vx[i] *= 1.001

    run = OracleStandIn(rp, st, ne, plant=(7, plant))
    t, _ = P.lockstep(run, rp, st, 10, ne_cells=ne, vel_rel=5e-5)
    assert t["vel"] >= 1 and t["first_bad"]["step"] == 7, t


def test_planted_charge_state_error_is_reported():
    rp, st, ne = setup(False)

    def plant(o):
        i = _far_ion(o, rp)
        o.q[i] += 1

    run = OracleStandIn(rp, st, ne, plant=(4, plant))
    t, _ = P.lockstep(run, rp, st, 6, ne_cells=ne)
    assert t["q"] >= 1 and t["first_bad"]["step"] == 4, t


def test_planted_pairing_error_is_reported():
    # two ions of one cell exchange their post-collision velocities: a wrong
    # pairing that no flagged decision explains
    rp, st, ne = setup(True)

    def plant(o):
        cells = P.ngp(rp, o)
        i = _far_ion(o, rp)
        same = np.nonzero((cells == cells[i]) & (o.q >= 1) & (np.arange(o.n) != i))[0]
        j = int(same[0])
        for k in ("vx", "vy", "vz"):
            a = getattr(o, k)
            a[i], a[j] = a[j], a[i]

    run = OracleStandIn(rp, st, ne, plant=(6, plant))
    t, _ = P.lockstep(run, rp, st, 8, ne_cells=ne, vel_rel=5e-5)
    assert t["vel"] >= 2 and t["first_bad"]["step"] == 6, t
