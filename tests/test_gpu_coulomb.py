"""GPU parity of the Coulomb collision kernels (Takizawa-Abe pairing, Nanbu
angle) with the FP64 oracle, through the C ABI.

Cells hold 1 to several thousand ions so that both the shared-memory path of
the collision kernel and its global-memory path (a range of cells larger than
shared memory holds) run, with ranges that split anywhere; every pairing
must be identical to the oracle's (integer events and collision counts) and
the velocities must agree to 5e-5 of |v|, the FP32 rounding of the collision
arithmetic with a margin.  The lock-step checker (tests/parity.py) compares
every particle; a particle that took the other side of a decision within
rounding of its surface, and the ions its flip re-paired, must match the
oracle's probe of that decision.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1507_03392_gb300 import inputs as I
from tests import parity as P

pytestmark = pytest.mark.gpu
QE = 1.602176634e-19
AMU = 1.66053906660e-27


@pytest.fixture(scope="module")
def E():
    from paper_1507_03392_gb300 import ecris
    return ecris


def cells_state(rp, sizes, seed, T_eV=0.5, qmax_init=10):
    """ions grouped at the centres of distinct cells, len(sizes) cells"""
    rng = np.random.default_rng(seed)
    dx, dy, dz = 2 * rp.R0 / rp.nx, 2 * rp.R0 / rp.ny, rp.L / rp.nz
    cells = rng.choice(np.arange(rp.nx * rp.ny * rp.nz), size=len(sizes), replace=False)
    xs, ys, zs = [], [], []
    for c, m in zip(cells, sizes):
        ix, iy, iz = c % rp.nx, (c // rp.nx) % rp.ny, c // (rp.nx * rp.ny)
        # spread inside the cell, away from its faces
        xs.append(-rp.R0 + (ix + rng.uniform(0.2, 0.8, m)) * dx)
        ys.append(-rp.R0 + (iy + rng.uniform(0.2, 0.8, m)) * dy)
        zs.append((iz + rng.uniform(0.2, 0.8, m)) * dz)
    x, y, z = (np.concatenate(a).astype(np.float32) for a in (xs, ys, zs))
    inside = x.astype(np.float64) ** 2 + y.astype(np.float64) ** 2 < 0.98 * rp.R0 ** 2
    n = len(x)
    sig = math.sqrt(T_eV * QE / (rp.species.mass_amu * AMU))
    v = rng.normal(0, sig, (3, n)).astype(np.float32)
    q = rng.integers(1, qmax_init + 1, n).astype(np.uint8)
    q[rng.random(n) < 0.1] = 0          # a few atoms take no part
    keep = inside
    return {"x": x[keep], "y": y[keep], "z": z[keep], "vx": v[0][keep], "vy": v[1][keep],
            "vz": v[2][keep], "q": q[keep]}


@pytest.mark.parametrize("sizes,seed", [([1, 2, 3, 7, 31, 32, 33], 1),
                                        ([40, 100, 511, 1024, 1025], 2),
                                        ([3000], 3)])
def test_coulomb_only_lockstep_all_sort_paths(E, sizes, seed):
    rp = I.RunParams(nx=8, ny=8, nz=16, flags=I.F_COULOMB, weight=5e7, dt=1e-8, seed=seed)
    st = cells_state(rp, sizes, seed)
    run = E.Run(rp)
    run.load(st)
    t, orc = P.lockstep(run, rp, st, 3, vel_rel=5e-5)
    assert t["q"] == 0 and t["events"] == 0 and t["pos"] == 0 and t["vel"] == 0, t
    d = run.diag()
    assert d["coulomb_collisions"] == orc.tally.coulomb_pairs
    run.close()


def test_coulomb_lockstep_on_a_mesh_of_many_scan_tiles(E):
    # 96 x 96 x 192 cells: the per-cell count scan runs 864 tiles of 2048
    # cells, so a tile's look-back over the totals before it (256 tiles a
    # round) may take several rounds; ions sit in cells spread over the whole
    # mesh, one of them above the shared-memory capacity of a range
    rp = I.RunParams(nx=96, ny=96, nz=192, flags=I.F_COULOMB, weight=5e7, dt=1e-8, seed=11)
    rng = np.random.default_rng(11)
    sizes = [int(m) for m in rng.integers(1, 40, 500)] + [1100]
    st = cells_state(rp, sizes, 11)
    run = E.Run(rp)
    run.load(st)
    t, orc = P.lockstep(run, rp, st, 3, vel_rel=5e-5)
    assert t["q"] == 0 and t["events"] == 0 and t["pos"] == 0 and t["vel"] == 0, t
    d = run.diag()
    assert d["coulomb_collisions"] == orc.tally.coulomb_pairs
    assert d["coulomb_collisions"] > 3000
    run.close()


def test_coulomb_conserves_momentum_and_energy_per_cell(E):
    rp = I.RunParams(nx=8, ny=8, nz=16, flags=I.F_COULOMB, weight=2e8, dt=2e-8, seed=5)
    sizes = [2, 5, 64, 300, 2000]
    st = cells_state(rp, sizes, 5, T_eV=2.0)
    run = E.Run(rp)
    run.load(st)
    g0 = run.state()
    run.step(1)
    g1 = run.state()
    dx, dy, dz = 2 * rp.R0 / rp.nx, 2 * rp.R0 / rp.ny, rp.L / rp.nz
    cell = ((np.floor(g0["z"] / dz) * rp.ny + np.floor((g0["y"] + rp.R0) / dy)) * rp.nx
            + np.floor((g0["x"] + rp.R0) / dx)).astype(np.int64)
    moved = 0
    for c in np.unique(cell):
        sel = (cell == c) & (g0["q"] >= 1)
        v0 = np.stack([g0[k][sel] for k in ("vx", "vy", "vz")]).astype(np.float64)
        v1 = np.stack([g1[k][sel] for k in ("vx", "vy", "vz")]).astype(np.float64)
        scale = np.abs(v0).sum()
        assert np.abs(v0.sum(axis=1) - v1.sum(axis=1)).max() <= 1e-5 * scale + 1e-3
        assert (v1 ** 2).sum() == pytest.approx((v0 ** 2).sum(), rel=1e-5)
        moved += int((np.abs(v1 - v0).max(axis=0) > 0).sum())
    assert moved > 0.8 * int((g0["q"] >= 1).sum())
    run.close()


def test_full_step_with_coulomb_lockstep(E):
    # every process on, ions dense enough for many multi-ion cells
    rp = I.RunParams(nx=16, ny=16, nz=32, ne_in_cm3=2e12, ne_out_cm3=2e11, n0_cm3=2e11, dt=2e-8,
                     flags=I.F_ALL, weight=1e8, seed=8)
    wl = I.Workload("dense", rp, n=20000, steps=0, atom_fraction=0.3, ion_qmax_init=8, ion_T_eV=5.0,
                    atoms_fill_chamber=True, zone_box=(0.01, 0.17, 0.2))
    st = I.make_particles(wl, seed=8)
    Ef = I.make_efield(rp, 2e3, -1e3)
    run = E.Run(rp, E=Ef)
    run.load(st)
    t, orc = P.lockstep(run, rp, st, 8, E=Ef, vel_rel=5e-5)
    assert t["q"] == 0 and t["events"] == 0 and t["pos"] == 0 and t["vel"] == 0, (t, t["first_bad"])
    assert t["guarded_frac"] < 0.02 and t["accepted_frac"] < 0.01, t
    d = run.diag()
    assert d["coulomb_collisions"] > 1000
    run.close()


def test_hot_ions_small_angles_lockstep(E):
    # Hot oxygen ions packed into few cells: fast relative velocities make
    # most collisions small-angle ones, where cos chi lies within FP32
    # rounding of 1.  The kernel forms 1 - cos chi and sin chi without
    # cancellation, so the velocities follow the FP64 oracle to 5e-5 of |v|.
    # The longest sort cadence lets the ions drift far from the cells they
    # were grouped by, and particles that reach the wall are frozen (no
    # recycling).
    rp = I.RunParams(species=I.OXYGEN, nx=16, ny=16, nz=32, flags=I.F_PUSH | I.F_COULOMB, weight=5e7,
                     dt=2e-8, seed=31)
    wl = I.Workload("hot_packed", rp, n=20000, steps=0, atom_fraction=0.05, ion_qmax_init=4, ion_T_eV=20.0,
                    zone_box=(0.009, 0.14, 0.16))
    st = I.make_particles(wl, seed=31)
    run = E.Run(rp)
    run.set_tuning(sort_every=128)
    run.load(st)
    t, orc = P.lockstep(run, rp, st, 60, vel_rel=5e-5)
    assert t["q"] == 0 and t["events"] == 0 and t["pos"] == 0 and t["vel"] == 0, (t, t["first_bad"])
    d = run.diag()
    assert d["coulomb_collisions"] == orc.tally.coulomb_pairs
    run.close()


def test_thousand_steps_every_process_with_coulomb_lockstep(E):
    # 2e4 particles, every process on (push with an E grid, ionisation, charge
    # exchange, heating kick, recycling, ion-ion collisions), 1000 steps in
    # lock-step: every particle is compared at every step; the few that took
    # the other side of a decision within rounding of its surface must match
    # the oracle's probe of that decision
    rp = I.RunParams(nx=16, ny=16, nz=32, ne_in_cm3=1e12, ne_out_cm3=1e11, n0_cm3=1e11, dt=1e-8,
                     flags=I.F_ALL, weight=1e8, seed=12)
    wl = I.Workload("dense_1000", rp, n=20000, steps=0, atom_fraction=0.4, ion_qmax_init=8, ion_T_eV=2.0,
                    atoms_fill_chamber=True, zone_box=(0.012, 0.15, 0.2))
    st = I.make_particles(wl, seed=12)
    Ef = I.make_efield(rp, 2e3, -1e3)
    run = E.Run(rp, E=Ef)
    run.load(st)
    t, orc = P.lockstep(run, rp, st, 1000, E=Ef, vel_rel=5e-5)
    print(f"\n[Coulomb on, 2e4 particles, 1000 steps] events seen (wall, extract, ionise, cx, coulomb): "
          f"{t['events_seen_all'][:5]}; flagged near a decision surface: {t['guarded_frac']:.2e} of "
          f"particle-steps; other side taken (explained by the probes): {t['accepted']} "
          f"({t['accepted_frac']:.1e})")
    assert t["q"] == 0 and t["events"] == 0 and t["pos"] == 0 and t["vel"] == 0, (t, t["first_bad"])
    assert t["guarded_frac"] < 0.02 and t["accepted_frac"] < 1e-3, t
    wall, ext, ion, cx, coul = t["events_seen_all"][:5]
    assert wall > 100 and ion > 100 and cx > 30 and coul > 1e6, t["events_seen_all"]
    d = run.diag()
    assert abs(d["coulomb_collisions"] - orc.tally.coulomb_pairs) <= 2 * t["accepted"]
    run.close()


def tied_hash_pids(seed, step=0, n_search=1 << 18):
    """two particle ids whose pairing hashes (stream-1 word 0 at `step`, the
    oracle's Philox) are equal: the pairing order then falls to the ids"""
    lo, hi = seed & 0xFFFFFFFF, seed >> 32
    seen = {}
    for pid in range(n_search):
        h = int(O.philox([pid, 0, 4 * step + 1, 0], [lo, hi])[0])
        if h in seen:
            return seen[h], pid
        seen[h] = pid
    return None


def test_tied_pairing_hashes_order_by_id(E):
    # two ions of one cell whose 32-bit pairing hashes are equal (about one
    # pair in 2^32): the kernel ranks by the hash words first and must fall
    # back to the whole key (hash, id) for that cell, as the oracle orders
    seed = 77
    pair = tied_hash_pids(seed)
    assert pair is not None
    p1, p2 = pair
    rp = I.RunParams(nx=8, ny=8, nz=16, flags=I.F_COULOMB, weight=5e7, dt=1e-8, seed=seed)
    n = p2 + 1
    rng = np.random.default_rng(5)
    dx, dz = 2 * rp.R0 / rp.nx, rp.L / rp.nz
    # atoms (no part in collisions) spread over the chamber's inner cells
    x = rng.uniform(-0.5, 0.5, n) * rp.R0
    y = rng.uniform(-0.5, 0.5, n) * rp.R0
    z = rng.uniform(0.1, 0.9, n) * rp.L
    q = np.zeros(n, dtype=np.uint8)
    # five ions in one cell: the tied pair and three others, an odd count so
    # that the order decides the triplet and the pair
    ions = [p1, p2, 0, 1, 2] if p1 > 2 else [p1, p2, n - 1, n - 2, n - 3]
    cx, cy, cz = 3, 4, 7
    for k, p in enumerate(ions):
        x[p] = -rp.R0 + (cx + 0.3 + 0.1 * k) * dx
        y[p] = -rp.R0 + (cy + 0.5) * dx
        z[p] = (cz + 0.5) * dz
        q[p] = 3
    sig = math.sqrt(0.5 * QE / (rp.species.mass_amu * AMU))
    v = rng.normal(0, sig, (3, n))
    st = {"x": x.astype(np.float32), "y": y.astype(np.float32), "z": z.astype(np.float32),
          "vx": v[0].astype(np.float32), "vy": v[1].astype(np.float32), "vz": v[2].astype(np.float32), "q": q}
    run = E.Run(rp)
    run.load(st)
    t, orc = P.lockstep(run, rp, st, 1, vel_rel=5e-5)
    assert t["q"] == 0 and t["events"] == 0 and t["pos"] == 0 and t["vel"] == 0, t
    assert run.diag()["coulomb_collisions"] == orc.tally.coulomb_pairs == 4
    run.close()
