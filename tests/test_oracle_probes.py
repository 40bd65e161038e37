"""Pins of the oracle's diagnostics of Sec. III.A: moment probes (densities,
temperatures, ion pressure), screen images and the mean radial displacement
of the extracted ions, against closed forms of constructed states."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1507_03392_gb300 import inputs as I

QE, AMU = 1.602176634e-19, 1.66053906660e-27


def _centre(rp, ix, iy, iz):
    dx, dy, dz = 2 * rp.R0 / rp.nx, 2 * rp.R0 / rp.ny, rp.L / rp.nz
    return -rp.R0 + (ix + 0.5) * dx, -rp.R0 + (iy + 0.5) * dy, (iz + 0.5) * dz


def _state(rows):
    """rows of (x, y, z, vx, vy, vz, q)"""
    a = np.array(rows, dtype=np.float64).reshape(-1, 7)
    st = {k: a[:, i].copy() for i, k in enumerate(("x", "y", "z", "vx", "vy", "vz"))}
    st["q"] = a[:, 6].astype(np.int32)
    return st


def test_six_beam_cell_has_closed_form_temperature():
    # six ions of charge 3 moving +-a along each axis: <v> = 0, <v^2> = a^2,
    # so T = M a^2 / 3 and P = n T with n = 6 w / V; plus a drifting pair of
    # charge 5 (v = u +- b along x): T = M b^2 / 3, the drift does not count
    rp = I.RunParams(nx=8, ny=8, nz=16, weight=2e8)
    a, u, b = 2.0e4, 7.0e3, 3.0e3
    cx, cy, cz = _centre(rp, 3, 4, 9)
    rows = [(cx, cy, cz, s * a * (k == 0), s * a * (k == 1), s * a * (k == 2), 3)
            for k in range(3) for s in (1, -1)]
    rows += [(cx, cy, cz, u + b, 0, 0, 5), (cx, cy, cz, u - b, 0, 0, 5)]
    # a particle in another (unprobed) cell changes nothing
    ox, oy, oz = _centre(rp, 2, 4, 9)
    rows.append((ox, oy, oz, 1e5, 0, 0, 3))
    st = _state(rows)
    c = (9 * rp.ny + 4) * rp.nx + 3
    mom = O.probe_moments(rp, st, [c])
    assert mom[0, 3, 0] == 6 and mom[0, 5, 0] == 2 and mom[0].sum(axis=0)[0] == 8
    assert np.allclose(mom[0, 3, 4:], 2 * a * a) and np.allclose(mom[0, 3, 1:4], 0)
    prof = O.moment_profiles(rp, 2 * mom, samples=2)   # two identical samples
    M = rp.species.mass_amu * AMU
    vol = (2 * rp.R0 / rp.nx) * (2 * rp.R0 / rp.ny) * (rp.L / rp.nz)
    assert prof["T_eV"][0, 3] == pytest.approx(M * a * a / 3 / QE, rel=1e-12)
    assert prof["T_eV"][0, 5] == pytest.approx(M * b * b / 3 / QE, rel=1e-9)
    n3, n5 = 6 * rp.weight / vol, 2 * rp.weight / vol
    assert prof["n"][0, 3] == pytest.approx(n3, rel=1e-12)
    P = n3 * M * a * a / 3 / QE + n5 * M * b * b / 3 / QE
    assert prof["P_eV_m3"][0] == pytest.approx(P, rel=1e-9)
    assert prof["T_mean_eV"][0] == pytest.approx(P / (n3 + n5), rel=1e-9)


def test_maxwellian_temperature_within_sampling_error():
    rp = I.RunParams(nx=8, ny=8, nz=16)
    rng = np.random.default_rng(3)
    T_eV, N = 25.0, 40000
    M = rp.species.mass_amu * AMU
    sig = np.sqrt(T_eV * QE / M)
    cx, cy, cz = _centre(rp, 4, 4, 8)
    st = {"x": np.full(N, cx), "y": np.full(N, cy), "z": np.full(N, cz),
          "vx": rng.normal(0, sig, N), "vy": rng.normal(0, sig, N), "vz": rng.normal(500.0, sig, N),
          "q": np.full(N, 2, dtype=np.int32)}
    c = (8 * rp.ny + 4) * rp.nx + 4
    prof = O.moment_profiles(rp, O.probe_moments(rp, st, [c]), samples=1)
    # the estimate's relative standard deviation is about sqrt(2 / (3 N))
    assert abs(prof["T_eV"][0, 2] / T_eV - 1) < 5 * np.sqrt(2 / (3 * N))


def test_screen_counts_pixels_and_slab_edges():
    rp = I.RunParams(nx=8, ny=8, nz=16)
    P = 16
    pw = 2 * rp.R0 / P
    lo, hi = 0.165, 0.175
    rows = []
    want = np.zeros((1, rp.species.qmax + 1, P, P), dtype=np.int64)
    rng = np.random.default_rng(5)
    for _ in range(300):
        px, py = rng.integers(2, P - 2, size=2)
        q = int(rng.integers(0, 9))
        z = rng.uniform(lo, hi)
        rows.append((-rp.R0 + (px + 0.5) * pw, -rp.R0 + (py + 0.5) * pw, z, 0, 0, 0, q))
        want[0, q, py, px] += 1
    # on the lower slab face: in; on the upper face and outside: out
    rows.append((-rp.R0 + 5.5 * pw, -rp.R0 + 6.5 * pw, lo, 0, 0, 0, 1))
    want[0, 1, 6, 5] += 1
    rows.append((-rp.R0 + 5.5 * pw, -rp.R0 + 6.5 * pw, hi, 0, 0, 0, 1))
    rows.append((0.0, 0.0, 0.1, 0, 0, 0, 1))
    got = O.screen_hits(rp, _state(rows), [(lo, hi)], P)
    assert np.array_equal(got, want)


def test_extraction_radius_of_straight_atoms():
    # atoms move straight along z: each crosses the aperture plane where it
    # started in x-y, so the summed radius is the sum of the start radii
    rp = I.RunParams(nx=8, ny=8, nz=16, flags=I.F_PUSH | I.F_RECYCLE, dt=1e-8)
    rng = np.random.default_rng(8)
    n = 200
    r = 0.95 * rp.r_ap * np.sqrt(rng.random(n))
    ph = 2 * np.pi * rng.random(n)
    st = {"x": r * np.cos(ph), "y": r * np.sin(ph), "z": rp.L - rng.uniform(0.001, 0.02, n),
          "vx": np.zeros(n), "vy": np.zeros(n), "vz": np.full(n, 3e4), "q": np.zeros(n, dtype=np.int32)}
    o = O.OracleRun(rp, st)
    o.step(80)
    assert o.extracted()[0] == n
    assert o.tally.r_ext_sum[0] == pytest.approx(r.sum(), rel=1e-12)
    assert o.tally.r_ext_sum[1] == 0.0
