"""Pins of the oracle's field model and E-grid gather.

Paper: Sec. II, the B_x/B_y equations (hexapole added analytically to the
solenoid field, B_H at the chamber wall R0) and the statement that the
longitudinal field comes from axisymmetric solenoids (Figs. 2-3, extremes
B_inj, B_min, B_ext).  The synthetic mirror profile, the paraxial expansion and
the cell-centred trilinear E gather are the readings stated in the design notes.
"""
import ctypes
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1507_03392_gb300 import inputs as I


@pytest.fixture
def p():
    return O.make_params(I.RunParams())


def test_axial_profile_extremes(p):
    zm = O.lib().or_zmin(ctypes.byref(p))
    assert O.b0(p, 0.0)[0] == pytest.approx(p.B_inj, rel=1e-14)
    assert O.b0(p, zm)[0] == pytest.approx(p.B_min, rel=1e-14)
    assert O.b0(p, p.L)[0] == pytest.approx(p.B_ext, rel=1e-14)
    # the minimum is a true minimum, with zero slope at the extremes
    zs = np.linspace(0, p.L, 3001)
    vals = np.array([O.b0(p, z)[0] for z in zs])
    assert vals.min() >= p.B_min - 1e-12
    for z in (0.0, zm, p.L):
        assert abs(O.b0(p, z)[1]) < 1e-9
    # z_m near the paper's B_min location for KVI-like fields (z ~ 17-18 cm)
    assert 0.17 < zm < 0.19


def test_axial_profile_derivatives_and_continuity(p):
    zm = O.lib().or_zmin(ctypes.byref(p))
    h = 1e-6
    for z in np.linspace(0.01, p.L - 0.01, 37):
        b = O.b0(p, z)
        d1 = (O.b0(p, z + h)[0] - O.b0(p, z - h)[0]) / (2 * h)
        d2 = (O.b0(p, z + h)[1] - O.b0(p, z - h)[1]) / (2 * h)
        assert b[1] == pytest.approx(d1, rel=1e-6, abs=1e-6)
        assert b[2] == pytest.approx(d2, rel=1e-5, abs=1e-4)
    # B0'' continuous across the joint at z_m (the condition that fixes z_m)
    left = O.b0(p, zm - 1e-12)[2]
    right = O.b0(p, zm + 1e-12)[2]
    assert left == pytest.approx(right, rel=1e-9)


def test_hexapole_magnitude_and_printed_components(p):
    # pure hexapole: no solenoid (B_inj=B_min=B_ext would give a uniform Bz)
    q = O.make_params(I.RunParams(B_inj=0.0, B_min=0.0, B_ext=0.0))
    q.B_inj, q.B_min, q.B_ext = 1e-30, 0.0, 1e-30
    rng = np.random.default_rng(3)
    for _ in range(50):
        R = rng.uniform(0.001, q.R0)
        th = rng.uniform(0, 2 * math.pi)
        x, y = R * math.cos(th), R * math.sin(th)
        B = O.bfield(q, x, y, 0.15)
        assert math.hypot(B[0], B[1]) == pytest.approx(q.B_hex * (R / q.R0) ** 2, rel=1e-9)
        # printed form: B_x = B_H sin(2 theta) R^2/R0^2, B_y = B_H cos(2 theta) R^2/R0^2
        assert B[0] == pytest.approx(q.B_hex * math.sin(2 * th) * R * R / q.R0 ** 2, abs=1e-12)
        assert B[1] == pytest.approx(q.B_hex * math.cos(2 * th) * R * R / q.R0 ** 2, abs=1e-12)
    # |B_hex| at the wall equals B_H
    B = O.bfield(q, 0.0, q.R0, 0.15)
    assert math.hypot(B[0], B[1]) == pytest.approx(q.B_hex, rel=1e-12)


def _div_curl(p, x, y, z, h=1e-6):
    J = np.zeros((3, 3))
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        J[:, k] = (O.bfield(p, *(np.array([x, y, z]) + e)) - O.bfield(p, *(np.array([x, y, z]) - e))) / (2 * h)
    div = J[0, 0] + J[1, 1] + J[2, 2]
    curl = np.array([J[2, 1] - J[1, 2], J[0, 2] - J[2, 0], J[1, 0] - J[0, 1]])
    return div, curl


def test_hexapole_is_divergence_and_curl_free():
    q = O.make_params(I.RunParams())
    q.B_inj, q.B_min, q.B_ext = 1e-30, 0.0, 1e-30
    for (x, y) in [(0.01, 0.004), (-0.02, 0.013), (0.005, -0.025)]:
        div, curl = _div_curl(q, x, y, 0.1)
        assert abs(div) < 1e-6 and np.abs(curl).max() < 1e-6


def test_paraxial_solenoid_divergence_and_curl(p):
    # B_r = -(r/2) B0', B_z = B0 - (r^2/4) B0'': the curl vanishes and
    # div B = -(r^2/4) times the third derivative of B0 (second order in r)
    p.B_hex = 0.0
    h = 1e-5
    for z in (0.05, 0.12, 0.21, 0.27):
        b3 = (O.b0(p, z + h)[2] - O.b0(p, z - h)[2]) / (2 * h)
        for r in (0.002, 0.004, 0.008):
            div, curl = _div_curl(p, r * 0.6, r * 0.8, z)
            assert div == pytest.approx(-0.25 * r * r * b3, rel=1e-3, abs=1e-9)
            assert np.abs(curl).max() < 1e-6


def test_trilinear_gather_exact_for_linear_field():
    rp = I.RunParams(nx=8, ny=8, nz=16)
    p = O.make_params(rp)
    E = I.make_efield(rp, 1234.0, -567.0).astype(np.float64).reshape(-1)
    dx = 2 * rp.R0 / rp.nx
    dz = rp.L / rp.nz
    rng = np.random.default_rng(5)
    out = np.zeros(3)
    for _ in range(200):
        # stay between the first and last cell centres, where no clamping applies
        x = rng.uniform(-rp.R0 + dx / 2, rp.R0 - dx / 2)
        y = rng.uniform(-rp.R0 + dx / 2, rp.R0 - dx / 2)
        z = rng.uniform(dz / 2, rp.L - dz / 2)
        O.lib().or_efield(ctypes.byref(p), E.ctypes.data_as(ctypes.c_void_p), x, y, z,
                          out.ctypes.data_as(ctypes.c_void_p))
        assert out == pytest.approx([1234.0 * x, 1234.0 * y, -567.0 * (z - rp.L / 2)], rel=1e-5, abs=1e-3)
    # outside the outer centres the face value is held (clamped gather)
    O.lib().or_efield(ctypes.byref(p), E.ctypes.data_as(ctypes.c_void_p), -rp.R0 + dx / 4, 0.0,
                      rp.L / 2, out.ctypes.data_as(ctypes.c_void_p))
    assert out[0] == pytest.approx(1234.0 * (-rp.R0 + dx / 2), rel=1e-6)
