"""GPU test of ecris_coulomb_collide_noalloc, the allocation-free Coulomb step.

Some callers cannot allocate device memory when they need a collision step:
hosts that reserve all device memory up front, plug-ins whose memory manager
owns the device, code that must not let cudaMalloc synchronise the device.
They call ecris_coulomb_collide_noalloc, which keeps its working memory in a
fixed array inside the library.  These tests call it through the C ABI on two
consecutive steps and check each result against ecris_step with only the
Coulomb collisions switched on (the existing path).  Both run the same
pairing and the same collision arithmetic on the same FP64-built Nanbu table,
so the velocities must be identical bit for bit.  The cases reach the fixed
limits of the working array (65536 particles in 65536 cells, one cell larger
than the collision kernel's shared-memory range) and a single cell.  The file
is collected last by pytest.
"""
import ctypes
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
QE = 1.602176634e-19
AMU = 1.66053906660e-27


def grouped_ions(rp, sizes, seed, total=None, r_max=0.9):
    """ions at the centres of distinct cells (well inside the cylinder), len(sizes)
    cells of the given sizes; with `total`, exactly that many particles"""
    rng = np.random.default_rng(seed)
    dx, dy, dz = 2 * rp.R0 / rp.nx, 2 * rp.R0 / rp.ny, rp.L / rp.nz
    allc = np.arange(rp.nx * rp.ny * rp.nz)
    ix, iy = allc % rp.nx, (allc // rp.nx) % rp.ny
    # every point of the cell inside r_max R0
    fx = np.maximum(np.abs(-rp.R0 + ix * dx), np.abs(-rp.R0 + (ix + 1) * dx))
    fy = np.maximum(np.abs(-rp.R0 + iy * dy), np.abs(-rp.R0 + (iy + 1) * dy))
    inner = allc[fx ** 2 + fy ** 2 < (r_max * rp.R0) ** 2]
    cells = rng.choice(inner, size=len(sizes), replace=False)
    xs, ys, zs, cs = [], [], [], []
    for c, m in zip(cells, sizes):
        cx, cy, cz = c % rp.nx, (c // rp.nx) % rp.ny, c // (rp.nx * rp.ny)
        xs.append(-rp.R0 + (cx + rng.uniform(0.2, 0.8, m)) * dx)
        ys.append(-rp.R0 + (cy + rng.uniform(0.2, 0.8, m)) * dy)
        zs.append((cz + rng.uniform(0.2, 0.8, m)) * dz)
        cs.append(np.full(m, c, dtype=np.uint32))
    x, y, z = (np.concatenate(a).astype(np.float32) for a in (xs, ys, zs))
    cell = np.concatenate(cs)
    if total is not None:
        assert len(x) == total
    n = len(x)
    sig = math.sqrt(1.0 * QE / (rp.species.mass_amu * AMU))
    v = rng.normal(0, sig, (3, n)).astype(np.float32)
    q = rng.integers(1, 9, n).astype(np.uint8)
    q[rng.random(n) < 0.1] = 0
    st = {"x": x, "y": y, "z": z, "vx": v[0], "vy": v[1], "vz": v[2], "q": q}
    return st, cell


def run_both(rp, st, cell, ncells_arg=None):
    """two steps of ecris_step (collisions only) and two calls of the
    allocation-free entry point on the same state; velocities, collision
    flags and counts must agree exactly"""
    import torch

    from paper_1507_03392_gb300 import ecris as E

    n = len(st["x"])
    run = E.Run(rp)
    run.load(st)
    dev = torch.device("cuda", 0)
    t_cell = torch.from_numpy(cell.view(np.int32)).to(dev)
    t_q = torch.from_numpy(st["q"]).to(dev)
    t_v = [torch.from_numpy(st[k].copy()).to(dev) for k in ("vx", "vy", "vz")]
    t_ev = torch.zeros(n, dtype=torch.int32, device=dev)
    vol = (2 * rp.R0 / rp.nx) * (2 * rp.R0 / rp.ny) * (rp.L / rp.nz)
    ncells = rp.nx * rp.ny * rp.nz if ncells_arg is None else ncells_arg
    stream = torch.cuda.current_stream().cuda_stream
    prev = 0
    for step in (0, 1):
        run.step(1)
        g = run.state()
        coll = ctypes.c_int64(0)
        status = E.ecris_coulomb_collide_noalloc(
            n, t_cell.data_ptr(), t_q.data_ptr(), t_v[0].data_ptr(), t_v[1].data_ptr(), t_v[2].data_ptr(),
            t_ev.data_ptr(), ncells, rp.species.mass_amu, rp.weight, vol, rp.lnL_ii, rp.dt,
            rp.seed, step, stream, ctypes.byref(coll))
        assert status == E.ECRIS_OK, E.ecris_last_error(None)
        torch.cuda.synchronize()
        for k, t in zip(("vx", "vy", "vz"), t_v):
            got = t.cpu().numpy()
            diff = np.abs(got.astype(np.float64) - g[k])
            assert np.array_equal(got, g[k]), (step, k, int((diff > 0).sum()), float(diff.max()))
        collided = (t_ev.cpu().numpy() & E.EV_COULOMB) != 0
        assert np.array_equal(collided, (g["meta"] & E.EV_COULOMB) != 0)
        total = run.diag()["coulomb_collisions"]
        assert coll.value == total - prev and coll.value > 0
        prev = total
        t_ev.zero_()
    run.close()


def test_noalloc_matches_ecris_step_on_two_calls():
    from paper_1507_03392_gb300 import inputs as I
    rp = I.RunParams(nx=16, ny=16, nz=32, flags=I.F_COULOMB, weight=5e7, dt=1e-8, seed=21)
    st, cell = grouped_ions(rp, [1, 2, 3, 9, 32, 33, 64, 65, 200, 700], seed=21)
    run_both(rp, st, cell)


def test_noalloc_at_its_limits_with_an_oversized_cell():
    # 65536 particles in a 65536-cell mesh, one cell of 1500 ions (above the
    # 1024 a collision range holds in shared memory: the global-memory path
    # and its sorted-position scratch)
    from paper_1507_03392_gb300 import inputs as I
    rp = I.RunParams(nx=32, ny=32, nz=64, flags=I.F_COULOMB, weight=5e7, dt=1e-8, seed=22)
    sizes = [1500] + [32] * 2000 + [36]
    assert sum(sizes) == 65536
    st, cell = grouped_ions(rp, sizes, seed=22, total=65536)
    run_both(rp, st, cell)


def test_noalloc_single_cell():
    # ncells = 1: every ion in cell 0; ecris_step sees the same ions in cell 0
    # of a 2x2x2 mesh (same cell volume)
    from paper_1507_03392_gb300 import inputs as I
    rp = I.RunParams(nx=2, ny=2, nz=2, flags=I.F_COULOMB, weight=5e7, dt=1e-8, seed=23)
    rng = np.random.default_rng(23)
    n = 301
    # cell 0 of the 2x2x2 mesh: x, y in [-R0, 0), z in [0, L/2); inside r < R0
    r = rp.R0 * np.sqrt(rng.uniform(0.05, 0.8, n))
    ph = rng.uniform(np.pi + 0.1, 1.5 * np.pi - 0.1, n)
    sig = math.sqrt(1.0 * QE / (rp.species.mass_amu * AMU))
    v = rng.normal(0, sig, (3, n)).astype(np.float32)
    q = rng.integers(1, 9, n).astype(np.uint8)
    st = {"x": (r * np.cos(ph)).astype(np.float32), "y": (r * np.sin(ph)).astype(np.float32),
          "z": rng.uniform(0.1, 0.4, n).astype(np.float32) * rp.L, "vx": v[0], "vy": v[1], "vz": v[2], "q": q}
    run_both(rp, st, np.zeros(n, dtype=np.uint32), ncells_arg=1)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_1507_03392_gb300 import ecris as E
    coll = ctypes.c_int64(0)
    status = E.ecris_coulomb_collide_noalloc(70000, 1, 1, 1, 1, 1, 1, 1024, 40.0, 1e8, 1e-8, 10.0, 1e-9,
                                             1, 0, None, ctypes.byref(coll))
    assert status == E.ECRIS_EINVAL
    assert b"65536" in E.ecris_last_error(None)
