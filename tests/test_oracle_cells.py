"""Pins of the oracle's per-cell electron data (Sec. II): warm electrons in the
ECR zone (|B| < B_ECR), cold outside; the delta vector of the electron
diamagnetic drift from the printed 3x3 stencil scaled by R_L."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1507_03392_gb300 import inputs as I


def _run(rp, ne_cells=None):
    st = {k: np.zeros(1) for k in ("x", "y", "vx", "vy", "vz")}
    st["z"] = np.full(1, 0.1)
    st["q"] = np.zeros(1, dtype=np.int32)
    return O.OracleRun(rp, st, ne_cells=ne_cells, deposit=False)


def test_delta_on_linear_ramp_matches_closed_form():
    # n(ix, iy) = n0 + gx ix + gy iy in every cell (B_ecr high: all cells warm).
    # For a linear ramp the stencil sums give -4 gy and 4 gx, so
    # delta = (4 R_L gy / n, -4 R_L gx / n) inside, half of that at an edge.
    rp = I.RunParams(B_ecr=100.0, nx=12, ny=12, nz=6)
    nc = rp.ncells
    ix = np.arange(nc) % rp.nx
    iy = (np.arange(nc) // rp.nx) % rp.ny
    n0, gx, gy = 3e11, 1.5e10, -0.8e10
    ne = (n0 + gx * ix + gy * iy).astype(np.float32)
    r = _run(rp, ne)
    dx = 2 * rp.R0 / rp.nx
    RL = 2.38e-6 * math.sqrt(rp.Te_warm_eV) / (r.Bmag * dx)
    nn = ne.astype(np.float64)
    inner = (ix > 0) & (ix < rp.nx - 1) & (iy > 0) & (iy < rp.ny - 1)
    assert np.allclose(r.dlx[inner], (4 * RL * gy / nn)[inner], rtol=1e-6)
    assert np.allclose(r.dly[inner], (-4 * RL * gx / nn)[inner], rtol=1e-6)
    # x edges (iy interior): the x-difference sees one clamped neighbour
    edge = (ix == 0) & (iy > 0) & (iy < rp.ny - 1)
    assert np.allclose(r.dly[edge], (-2 * RL * gx / nn)[edge], rtol=1e-6)
    assert np.allclose(r.dlx[edge], (4 * RL * gy / nn)[edge], rtol=1e-6)


def test_uniform_density_has_no_delta_and_zero_density_guard():
    rp = I.RunParams(B_ecr=100.0, nx=8, ny=8, nz=4)
    r = _run(rp)
    assert np.all(r.dlx == 0) and np.all(r.dly == 0)
    rp = I.RunParams(nx=8, ny=8, nz=4, ne_out_cm3=0.0)
    r = _run(rp)
    out = r.zone == 0
    assert np.all(r.ne[out] == 0) and np.all(r.dlx[out] == 0) and np.all(r.dly[out] == 0)


def test_zone_and_densities():
    rp = I.RunParams()
    r = _run(rp)
    assert np.all((r.Bmag < rp.B_ecr) == (r.zone == 1))
    assert np.all(r.ne[r.zone == 1] == pytest.approx(rp.ne_in_cm3 * 1e6))
    assert np.all(r.ne[r.zone == 0] == pytest.approx(rp.ne_out_cm3 * 1e6))
    # the zone is closed: it touches neither the flanges nor the side wall
    nz3 = r.zone.reshape(rp.nz, rp.ny, rp.nx)
    assert nz3[0].sum() == 0 and nz3[-1].sum() == 0
    assert nz3[:, 0, :].sum() == 0 and nz3[:, :, 0].sum() == 0
    assert 0.01 < r.zone.mean() < 0.1
