"""GPU parity of the diagnostics of Sec. III.A through the C ABI: moment
probes and screen images against the oracle's definitions applied to the
same particles, and the summed extraction radius against closed forms and
the oracle in lock-step."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1507_03392_gb300 import inputs as I
from tests import parity as P
from tests import test_gpu_fptd as F

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def E():
    from paper_1507_03392_gb300 import ecris
    return ecris


def _ulps(v):
    v = np.asarray(v, dtype=np.float32)
    return np.abs(np.spacing(v)).astype(np.float64)


def _near_faces(coord, origin, step, margin):
    """True where coord lies within margin of a face origin + k step."""
    t = (np.asarray(coord, np.float64) - origin) / step
    return np.abs(t - np.rint(t)) * step < margin


def _dirty(rp, st, slabs, pixels):
    """Particles whose cell, pixel or slab membership the FP32 export of a
    fixed-point position cannot decide (within 4 FP32 ulps of a face)."""
    x, y, z = (np.asarray(st[k], np.float32) for k in ("x", "y", "z"))
    mx, my, mz = 4 * _ulps(x) + 1e-10, 4 * _ulps(y) + 1e-10, 4 * _ulps(z) + 1e-10
    dx, dy, dz = 2 * rp.R0 / rp.nx, 2 * rp.R0 / rp.ny, rp.L / rp.nz
    cell = _near_faces(x, -rp.R0, dx, mx) | _near_faces(y, -rp.R0, dy, my) | _near_faces(z, 0.0, dz, mz)
    pw = 2 * rp.R0 / pixels
    pix = _near_faces(x, -rp.R0, pw, mx) | _near_faces(y, -rp.R0, pw, my)
    slab = np.zeros(len(x), dtype=bool)
    for lo, hi in slabs:
        slab |= (np.abs(z - lo) < mz) | (np.abs(z - hi) < mz)
    return cell, pix | slab


def _compare_moments(rp, got, want, bad_cells, cells):
    keep = ~np.isin(np.asarray(cells), bad_cells)
    assert keep.sum() >= 0.9 * len(cells)
    g, w = got[keep], want[keep]
    assert np.array_equal(g[..., 0], w[..., 0])
    scale = np.abs(w).max(axis=(0, 1)) + 1e-30
    assert np.all(np.abs(g - w) <= 1e-12 * scale + 1e-12 * np.abs(w))


def test_resting_particles_exact(E):
    rp = I.RunParams(nx=16, ny=16, nz=32, flags=0, weight=1e8)
    wl = I.Workload("p", rp, n=20001, steps=0, atom_fraction=0.3, ion_qmax_init=12, ion_T_eV=50.0,
                    atoms_fill_chamber=True)
    st = I.make_particles(wl, seed=3)
    slabs, px = [(0.165, 0.175), (0.29, rp.L)], 64
    cd, sd = _dirty(rp, st, slabs, px)
    keep = ~(cd | sd)
    st = {k: np.asarray(v)[keep] for k, v in st.items()}
    cells = np.unique(O.ngp_cells(rp, st["x"], st["y"], st["z"]))[::3]
    run = E.Run(rp)
    run.load(st)
    run.set_probes(cells, slabs, px)
    for _ in range(3):
        run.probe_sample()
        run.step(1)              # flags 0: nothing moves
    g = run.probes()
    assert g["samples"] == 3
    want = 3 * O.probe_moments(rp, st, cells)
    _compare_moments(rp, g["moments"], want, [], cells)
    assert np.array_equal(g["screens"].astype(np.int64), 3 * O.screen_hits(rp, st, slabs, px))
    assert g["screens"].sum() > 100
    # a load zeroes the sums; new probes replace the old ones
    run.load(st)
    assert run.probes()["samples"] == 0 and run.probes()["moments"].sum() == 0
    run.set_probes(cells[:5])
    run.probe_sample()
    g = run.probes()
    _compare_moments(rp, g["moments"], O.probe_moments(rp, st, cells[:5]), [], cells[:5])
    with pytest.raises(E.EcrisError):
        run.set_probes([cells[0], cells[0]])
    with pytest.raises(E.EcrisError):
        run.set_probes(cells[:2], [(0.1, 0.2)], pixels=48)
    run.close()


def test_busy_run_against_oracle(E):
    rp = I.RunParams(nx=16, ny=16, nz=32, ne_in_cm3=3e12, ne_out_cm3=3e11, n0_cm3=3e11, dt=3e-8,
                     Te_warm_eV=500.0, flags=I.F_ALL, seed=17)
    wl = I.Workload("pb", rp, n=30001, steps=0, atom_fraction=0.4, ion_qmax_init=8, ion_T_eV=60.0,
                    atoms_fill_chamber=True, zone_box=(0.02, 0.05, 0.29))
    st = I.make_particles(wl, seed=17)
    slabs, px = [(0.165, 0.175), (0.28, rp.L)], 128
    run = E.Run(rp)
    run.load(st)
    cells = np.arange(0, rp.ncells, 7)
    run.set_probes(cells, slabs, px)
    run.step(40)
    run.probe_sample()
    g = run.probes()
    s = run.state()
    alive = (s["meta"] & (1 << 16)) == 0
    cd, sd = _dirty(rp, s, slabs, px)
    want_m = O.probe_moments(rp, s, cells, alive=alive)
    # cells that a near-face particle might belong to on the device: its own
    # and the 26 around it
    c0 = O.ngp_cells(rp, s["x"], s["y"], s["z"])[cd]
    iz, rem = np.divmod(c0, rp.nx * rp.ny)
    iy, ix = np.divmod(rem, rp.nx)
    bad = []
    for oz in (-1, 0, 1):
        for oy in (-1, 0, 1):
            for ox in (-1, 0, 1):
                bad.append(((np.clip(iz + oz, 0, rp.nz - 1) * rp.ny + np.clip(iy + oy, 0, rp.ny - 1)) * rp.nx
                            + np.clip(ix + ox, 0, rp.nx - 1)))
    _compare_moments(rp, g["moments"], want_m, np.concatenate(bad) if bad else [], cells)
    want_s = O.screen_hits(rp, s, slabs, px, alive=alive & ~sd)
    near_s = O.screen_hits(rp, s, slabs, px, alive=alive & sd)
    got_s = g["screens"].astype(np.int64)
    # every pixel holds the far-from-edge hits, plus at most the near ones
    # around it
    pad = np.pad(near_s, ((0, 0), (0, 0), (1, 1), (1, 1)))
    slack = np.zeros_like(near_s)
    for oy in (0, 1, 2):
        for ox in (0, 1, 2):
            slack = np.maximum(slack, pad[:, :, oy:oy + px, ox:ox + px])
    slack *= 9
    assert np.all(got_s >= want_s - slack) and np.all(got_s <= want_s + slack)
    assert np.abs(got_s - want_s).sum() <= 2 * near_s.sum()
    assert got_s.sum() > 1000
    run.close()


def test_extraction_radius_closed_form(E):
    rp = I.RunParams(nx=8, ny=8, nz=16, flags=I.F_PUSH | I.F_RECYCLE, dt=1e-8)
    rng = np.random.default_rng(8)
    n = 2000
    r = 0.95 * rp.r_ap * np.sqrt(rng.random(n))
    ph = 2 * np.pi * rng.random(n)
    st = {"x": (r * np.cos(ph)).astype(np.float32), "y": (r * np.sin(ph)).astype(np.float32),
          "z": (rp.L - rng.uniform(0.001, 0.02, n)).astype(np.float32), "vx": np.zeros(n, np.float32),
          "vy": np.zeros(n, np.float32), "vz": np.full(n, 3e4, np.float32), "q": np.zeros(n, np.uint8)}
    run = E.Run(rp)
    run.load(st)
    run.step(80)
    assert run.diag()["extracted"][0] == n
    rs = run.extraction_radius()
    r32 = np.hypot(st["x"].astype(np.float64), st["y"].astype(np.float64))
    # whole nanometres per event, start positions rounded to the fixed-point grid
    assert abs(rs[0] - r32.sum()) <= n * 1e-9
    assert rs[1:].sum() == 0
    run.close()


def test_extraction_radius_lockstep(E):
    rp, st = F.aperture_case(23, I.F_ALL_NO_COULOMB)
    run = E.Run(rp)
    run.load(st)
    t, orc = P.lockstep(run, rp, st, 120)
    assert t["q"] == 0 and t["events"] == 0, t["first_bad"]
    d = run.diag()
    rs = run.extraction_radius()
    q1 = rp.species.qmax + 1
    ro = np.array(orc.tally.r_ext_sum[:q1])
    same = d["extracted"] == orc.extracted()
    assert same[1] and d["extracted"][1] >= 50
    # per event: whole nanometres on the device, and the crossing point from
    # the FP32 hand-over of the start (amplified at grazing incidence)
    assert np.all(np.abs(rs - ro)[same] <= d["extracted"][same] * 1e-7)
    run.close()


def test_batch_probes_equal_run_alone(E):
    rp = I.RunParams(nx=16, ny=16, nz=32, ne_in_cm3=3e12, n0_cm3=3e11, dt=3e-8, flags=I.F_ALL, seed=19)
    wl = I.Workload("pq", rp, n=8001, steps=0, atom_fraction=0.4, ion_qmax_init=8, ion_T_eV=60.0,
                    atoms_fill_chamber=True, zone_box=(0.02, 0.05, 0.29))
    st = I.make_particles(wl, seed=19)
    cells = np.arange(0, rp.ncells, 5)
    slabs = [(0.1, 0.2)]
    run = E.Run(rp)
    run.load(st)
    run.set_probes(cells, slabs, 32)
    b = E.Batch()
    h = b.add(rp, st)
    b.set_probes(h, cells, slabs, 32)
    for _ in range(4):
        run.step(10)
        b.step(10)
        run.probe_sample()
        b.probe_sample(h)
    ga, gb = run.probes(), b.probes(h)
    assert ga["samples"] == gb["samples"] == 4
    _compare_moments(rp, gb["moments"], ga["moments"], [], cells)
    assert np.array_equal(ga["screens"], gb["screens"])
    assert np.array_equal(run.extraction_radius(), b.extraction_radius(h))
    b.close()
    run.close()
