"""Pins of the oracle's self-consistent electron density (Sec. II: the electron
density equals the ion charge density, by charge neutrality).  n_e of a cell
is w times the charge the cell collected per step since the previous update,
over the cell volume; delta follows from it through the 3x3 stencil and R_L.

The expected values come from the particle placement alone (the cell of each
particle by the floor of its coordinate), not from the oracle's deposit."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1507_03392_gb300 import inputs as I


def _volume(rp):
    return (2 * rp.R0 / rp.nx) * (2 * rp.R0 / rp.ny) * (rp.L / rp.nz)


def _centre(rp, ix, iy, iz):
    dx, dy, dz = 2 * rp.R0 / rp.nx, 2 * rp.R0 / rp.ny, rp.L / rp.nz
    return -rp.R0 + (ix + 0.5) * dx, -rp.R0 + (iy + 0.5) * dy, (iz + 0.5) * dz


def _resting(rp, cells_q):
    """Ions at rest at cell centres: cells_q is a list of ((ix, iy, iz), Q)."""
    n = len(cells_q)
    st = {k: np.zeros(n) for k in ("x", "y", "z", "vx", "vy", "vz")}
    st["q"] = np.zeros(n, dtype=np.int32)
    for i, ((ix, iy, iz), q) in enumerate(cells_q):
        st["x"][i], st["y"][i], st["z"][i] = _centre(rp, ix, iy, iz)
        st["q"][i] = q
    return st


def _cell_index(rp, ix, iy, iz):
    return (iz * rp.ny + iy) * rp.nx + ix


def test_resting_ions_give_charge_density_in_every_cell():
    # no process acts (flags 0): the ions stay where they are and each step
    # deposits their charge again, so n_e = w sum(Q) / V_cell exactly
    rp = I.RunParams(nx=8, ny=8, nz=16, flags=0, weight=3e7)
    rng = np.random.default_rng(11)
    cq = []
    for _ in range(200):
        # inside the cylinder: cells whose centre is well within R0
        while True:
            ix, iy = rng.integers(2, rp.nx - 2, size=2)
            cx, cy, _ = _centre(rp, ix, iy, 0)
            if cx * cx + cy * cy < (0.8 * rp.R0) ** 2:
                break
        cq.append(((int(ix), int(iy), int(rng.integers(1, rp.nz - 1))), int(rng.integers(1, 9))))
    r = O.OracleRun(rp, _resting(rp, cq))
    r.step(7)
    r.update_ne()
    want = np.zeros(rp.ncells)
    for (ix, iy, iz), q in cq:
        want[_cell_index(rp, ix, iy, iz)] += q
    want *= rp.weight / _volume(rp)
    assert np.allclose(r.ne, want, rtol=1e-13, atol=0)
    # cells without ions have no electrons and no drift bias
    empty = want == 0
    assert np.all(r.dlx[empty] == 0) and np.all(r.dly[empty] == 0)
    # a second update averages only the steps since the first: the same density
    r.step(3)
    r.update_ne()
    assert np.allclose(r.ne, want, rtol=1e-13, atol=0)
    with pytest.raises(ValueError):
        r.update_ne()


def test_charge_ramp_gives_closed_form_delta():
    # sum(Q) per cell = a + bx ix + by iy (all cells warm: B_ECR high), so n_e
    # is a linear ramp with gradients gx = w bx / V, gy = w by / V per cell and
    # delta = (4 R_L gy / n_e, -4 R_L gx / n_e) at interior cells
    rp = I.RunParams(B_ecr=100.0, nx=10, ny=10, nz=4, flags=0, weight=1e8)
    a, bx, by = 40, 3, -2
    cq = []
    inner = []
    for iz in range(rp.nz):
        for iy in range(rp.ny):
            for ix in range(rp.nx):
                cx, cy, _ = _centre(rp, ix, iy, iz)
                if cx * cx + cy * cy >= (0.95 * rp.R0) ** 2:
                    continue
                total = a + bx * ix + by * iy
                # split the cell's charge over ions of Q <= 9
                while total > 0:
                    q = min(9, total)
                    cq.append(((ix, iy, iz), q))
                    total -= q
    for iz in range(rp.nz):
        for iy in range(1, rp.ny - 1):
            for ix in range(1, rp.nx - 1):
                ok = all(
                    (_centre(rp, ix + i, iy + j, iz)[0] ** 2 + _centre(rp, ix + i, iy + j, iz)[1] ** 2
                     < (0.95 * rp.R0) ** 2) for i in (-1, 0, 1) for j in (-1, 0, 1))
                if ok:
                    inner.append(_cell_index(rp, ix, iy, iz))
    assert len(inner) > 50
    r = O.OracleRun(rp, _resting(rp, cq))
    r.step(2)
    r.update_ne()
    inner = np.array(inner)
    V = _volume(rp)
    ix = inner % rp.nx
    iy = (inner // rp.nx) % rp.ny
    n = rp.weight * (a + bx * ix + by * iy) / V
    assert np.allclose(r.ne[inner], n, rtol=1e-13)
    dx = 2 * rp.R0 / rp.nx
    RL = 2.38e-6 * math.sqrt(rp.Te_warm_eV) / (r.Bmag[inner] * dx)
    gx, gy = rp.weight * bx / V, rp.weight * by / V
    assert np.allclose(r.dlx[inner], 4 * RL * gy / n, rtol=1e-9)
    assert np.allclose(r.dly[inner], -4 * RL * gx / n, rtol=1e-9)


def test_moving_ion_is_time_averaged():
    # one ion on the axis moving along B (no force: v parallel to B there)
    # at one cell length per step: over k steps it sits one step in each of k
    # cells, so each of them gets n_e = w Q / (k V)
    rp = I.RunParams(nx=8, ny=8, nz=32, flags=I.F_PUSH, weight=5e8)
    dz = rp.L / rp.nz
    iz0, k, Q = 4, 12, 3
    st = {k_: np.zeros(1) for k_ in ("x", "y", "z", "vx", "vy", "vz")}
    st["z"][0] = (iz0 + 0.5) * dz
    st["vz"][0] = dz / rp.dt
    st["q"] = np.full(1, Q, dtype=np.int32)
    r = O.OracleRun(rp, st)
    r.step(k)
    r.update_ne()
    # x = y = 0 lies on the face between the two middle cells: floor picks ix = nx/2
    want = np.zeros(rp.ncells)
    for s in range(1, k + 1):
        iz = iz0 + s
        want[_cell_index(rp, rp.nx // 2, rp.ny // 2, iz)] = rp.weight * Q / (k * _volume(rp))
    assert np.count_nonzero(r.ne) == k
    assert np.allclose(r.ne, want, rtol=1e-13, atol=0)
