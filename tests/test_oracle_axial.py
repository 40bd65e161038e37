"""Pins of the oracle's on-axis field table (the boundary's alternative to the
synthetic mirror): a natural cubic spline through B0 samples, extended off
axis by the paraxial expansion.  SciPy's CubicSpline with natural end
conditions is the library reference."""
import dataclasses

import numpy as np
import pytest
from scipy.interpolate import CubicSpline

from oracle import oracle as O
from paper_1507_03392_gb300 import inputs as I


def _table_params(values, **kw):
    return dataclasses.replace(I.RunParams(**kw), B_axial=tuple(float(v) for v in values))


@pytest.mark.parametrize("n", [4, 9, 65, 513])
def test_spline_matches_scipy_natural_spline(n):
    rng = np.random.default_rng(n)
    rp0 = I.RunParams()
    y = 0.4 + 1.8 * rng.random(n)
    rp = _table_params(y)
    p = O.make_params(rp)
    zk = np.linspace(0.0, rp.L, n)
    cs = CubicSpline(zk, y, bc_type="natural")
    z = np.concatenate([np.linspace(0.0, rp.L, 997), zk])
    for zz in z:
        out = np.zeros(3)
        O.lib().or_b0(p, float(zz), out.ctypes.data)
        want = np.array([cs(zz), cs(zz, 1), cs(zz, 2)])
        scale = np.array([1.0, 1.0 / rp.L, 1.0 / rp.L ** 2]) * 2.2
        assert np.all(np.abs(out - want) <= 1e-10 * scale * max(1, n) ** 2), (zz, out, want)
    assert rp0.B_axial is None


def test_sampled_mirror_reproduces_the_mirror_and_its_zone():
    rp0 = I.RunParams(nx=16, ny=16, nz=32)
    p0 = O.make_params(rp0)
    z = np.linspace(0.0, rp0.L, 1025)
    y = np.array([O.b0(p0, zz)[0] for zz in z])
    rp = dataclasses.replace(rp0, B_axial=tuple(y))
    p = O.make_params(rp)
    for zz in np.linspace(0.001, rp.L - 0.001, 301):
        a, b = O.b0(p0, zz), O.b0(p, zz)
        # 1025 samples: the spline's error is O(h^4 B0'''') in B0, O(h^3) in B0'
        assert abs(a[0] - b[0]) < 1e-6 and abs(a[1] - b[1]) < 0.02
    # the ECR zones agree
    st = {k: np.zeros(1) for k in ("x", "y", "vx", "vy", "vz")}
    st["z"] = np.full(1, 0.1)
    st["q"] = np.zeros(1, dtype=np.int32)
    r0 = O.OracleRun(rp0, st, deposit=False)
    r1 = O.OracleRun(rp, st, deposit=False)
    assert np.array_equal(r0.zone, r1.zone)


def test_off_axis_field_is_paraxial():
    rp = _table_params(I.flat_axial_profile(I.RunParams(), n=257, flat=0.06))
    p = O.make_params(rp)
    for (x, y, z) in [(0.0, 0.0, 0.12), (0.004, -0.002, 0.05), (-0.01, 0.006, 0.25)]:
        b0 = np.zeros(3)
        O.lib().or_b0(p, z, b0.ctypes.data)
        B = O.bfield(p, x, y, z)
        r2 = x * x + y * y
        assert B[2] == pytest.approx(b0[0] - 0.25 * r2 * b0[2], rel=1e-12, abs=1e-15)
        if r2 == 0.0:
            assert B[0] == 0.0 and B[1] == 0.0


def test_flat_profile_has_a_longer_zone():
    # the flat profile keeps B0 near B_min over a longer stretch of the axis,
    # so more cells lie below B_ECR
    rp0 = I.RunParams(nx=16, ny=16, nz=64, B_min=0.45)
    rp = dataclasses.replace(rp0, B_axial=I.flat_axial_profile(rp0, n=513, flat=0.08))
    st = {k: np.zeros(1) for k in ("x", "y", "vx", "vy", "vz")}
    st["z"] = np.full(1, 0.1)
    st["q"] = np.zeros(1, dtype=np.int32)
    z0 = O.OracleRun(rp0, st, deposit=False).zone.sum()
    z1 = O.OracleRun(rp, st, deposit=False).zone.sum()
    assert z1 > 1.5 * z0 > 0
