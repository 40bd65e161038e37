"""GPU test of ecris_coulomb_collide_noalloc, the allocation-free Coulomb step.

Some callers cannot allocate device memory when they need a collision step:
hosts that reserve all device memory up front, plug-ins whose memory manager
owns the device, code that must not let cudaMalloc synchronise the device.
They call ecris_coulomb_collide_noalloc, which keeps its working memory in a
fixed array inside the library.  This test calls it through the C ABI on two
consecutive steps and checks each result against ecris_step with only the
Coulomb collisions switched on (the existing path), within the velocity
tolerance the other Coulomb parity tests use.  It lives in a file of its own
that pytest collects last.
"""
import ctypes
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
QE = 1.602176634e-19
AMU = 1.66053906660e-27


def grouped_ions(rp, sizes, seed):
    rng = np.random.default_rng(seed)
    dx, dy, dz = 2 * rp.R0 / rp.nx, 2 * rp.R0 / rp.ny, rp.L / rp.nz
    cells = rng.choice(np.arange(rp.nx * rp.ny * rp.nz), size=len(sizes), replace=False)
    xs, ys, zs = [], [], []
    for c, m in zip(cells, sizes):
        ix, iy, iz = c % rp.nx, (c // rp.nx) % rp.ny, c // (rp.nx * rp.ny)
        xs.append(-rp.R0 + (ix + rng.uniform(0.2, 0.8, m)) * dx)
        ys.append(-rp.R0 + (iy + rng.uniform(0.2, 0.8, m)) * dy)
        zs.append((iz + rng.uniform(0.2, 0.8, m)) * dz)
    x, y, z = (np.concatenate(a).astype(np.float32) for a in (xs, ys, zs))
    keep = x.astype(np.float64) ** 2 + y.astype(np.float64) ** 2 < 0.98 * rp.R0 ** 2
    n = int(keep.sum())
    sig = math.sqrt(1.0 * QE / (rp.species.mass_amu * AMU))
    v = rng.normal(0, sig, (3, n)).astype(np.float32)
    q = rng.integers(1, 9, n).astype(np.uint8)
    q[rng.random(n) < 0.1] = 0
    x, y, z = x[keep], y[keep], z[keep]
    ix = np.floor((x.astype(np.float64) + rp.R0) / dx).astype(np.int64)
    iy = np.floor((y.astype(np.float64) + rp.R0) / dy).astype(np.int64)
    iz = np.floor(z.astype(np.float64) / dz).astype(np.int64)
    cell = ((iz * rp.ny + iy) * rp.nx + ix).astype(np.uint32)
    st = {"x": x, "y": y, "z": z, "vx": v[0], "vy": v[1], "vz": v[2], "q": q}
    return st, cell


def test_noalloc_matches_ecris_step_on_two_calls():
    import torch

    from paper_1507_03392_gb300 import ecris as E
    from paper_1507_03392_gb300 import inputs as I

    rp = I.RunParams(nx=16, ny=16, nz=32, flags=I.F_COULOMB, weight=5e7, dt=1e-8, seed=21)
    st, cell = grouped_ions(rp, [1, 2, 3, 9, 32, 33, 64, 65, 200, 700], seed=21)
    n = len(st["x"])
    run = E.Run(rp)
    run.load(st)

    dev = torch.device("cuda", 0)
    t_cell = torch.from_numpy(cell.view(np.int32)).to(dev)
    t_q = torch.from_numpy(st["q"]).to(dev)
    t_v = [torch.from_numpy(st[k].copy()).to(dev) for k in ("vx", "vy", "vz")]
    t_ev = torch.zeros(n, dtype=torch.int32, device=dev)
    vol = (2 * rp.R0 / rp.nx) * (2 * rp.R0 / rp.ny) * (rp.L / rp.nz)
    stream = torch.cuda.current_stream().cuda_stream
    prev = 0
    for step in (0, 1):
        run.step(1)
        g = run.state()
        coll = ctypes.c_int64(0)
        status = E.ecris_coulomb_collide_noalloc(
            n, t_cell.data_ptr(), t_q.data_ptr(), t_v[0].data_ptr(), t_v[1].data_ptr(), t_v[2].data_ptr(),
            t_ev.data_ptr(), rp.nx * rp.ny * rp.nz, rp.species.mass_amu, rp.weight, vol, rp.lnL_ii, rp.dt,
            rp.seed, step, stream, ctypes.byref(coll))
        assert status == E.ECRIS_OK, E.ecris_last_error(None)
        torch.cuda.synchronize()
        vmag = np.sqrt(sum(g[k].astype(np.float64) ** 2 for k in ("vx", "vy", "vz")))
        floor = math.sqrt(rp.T0_eV * QE / (rp.species.mass_amu * AMU))
        for k, t in zip(("vx", "vy", "vz"), t_v):
            got = t.cpu().numpy().astype(np.float64)
            assert np.all(np.abs(got - g[k]) <= 2e-4 * (vmag + floor)), (step, k)
        collided = (t_ev.cpu().numpy() & E.EV_COULOMB) != 0
        assert np.array_equal(collided, (g["meta"] & E.EV_COULOMB) != 0)
        total = run.diag()["coulomb_collisions"]
        assert coll.value == total - prev and coll.value > 0
        prev = total
        t_ev.zero_()
    run.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_1507_03392_gb300 import ecris as E
    coll = ctypes.c_int64(0)
    status = E.ecris_coulomb_collide_noalloc(70000, 1, 1, 1, 1, 1, 1, 1024, 40.0, 1e8, 1e-8, 10.0, 1e-9,
                                             1, 0, None, ctypes.byref(coll))
    assert status == E.ECRIS_EINVAL
    assert b"65536" in E.ecris_last_error(None)
