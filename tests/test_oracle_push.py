"""Pins of the oracle's particle mover (Sec. II: standard PIC push of the ions in
the static field; atoms move in straight lines).  The push is the Boris scheme
(Boris 1970), whose discrete orbits have closed forms in uniform fields."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1507_03392_gb300 import inputs as I

QE = 1.602176634e-19
AMU = 1.66053906660e-27


def test_boris_uniform_b_rotation_and_energy():
    B = np.array([0.0, 0.0, 0.7])
    qm = 3 * QE / (40 * AMU)
    dt = 3e-8
    omega = qm * B[2]
    theta = 2 * math.atan(omega * dt / 2)   # exact Boris phase advance per step
    v = np.array([1200.0, -300.0, 55.0])
    speed = np.linalg.norm(v)
    vp0 = math.atan2(v[1], v[0])
    for n in range(1, 400):
        v = O.boris(qm, [0, 0, 0], B, dt, v)
        assert np.linalg.norm(v) == pytest.approx(speed, rel=1e-13)
        assert v[2] == pytest.approx(55.0, rel=1e-13)
        # positive charge in +z field turns clockwise
        phase = math.atan2(v[1], v[0])
        want = vp0 - n * theta
        assert math.remainder(phase - want, 2 * math.pi) == pytest.approx(0.0, abs=1e-9)


def test_boris_gyroradius_closed_form():
    B = np.array([0.0, 0.0, 0.4])
    qm = 8 * QE / (40 * AMU)
    dt = 1e-8
    theta = 2 * math.atan(qm * B[2] * dt / 2)
    v = np.array([3000.0, 0.0, 0.0])
    x = np.zeros(3)
    pts = []
    for _ in range(300):
        v = O.boris(qm, [0, 0, 0], B, dt, v)
        x = x + v * dt
        pts.append(x[:2].copy())
    pts = np.array(pts)
    R = 3000.0 * dt / (2 * math.sin(theta / 2))
    # the positions lie on one circle of radius R: fit its centre from three points
    a, b, c = pts[0], pts[37], pts[111]
    d = 2 * (a[0] * (b[1] - c[1]) + b[0] * (c[1] - a[1]) + c[0] * (a[1] - b[1]))
    ux = ((a @ a) * (b[1] - c[1]) + (b @ b) * (c[1] - a[1]) + (c @ c) * (a[1] - b[1])) / d
    uy = ((a @ a) * (c[0] - b[0]) + (b @ b) * (a[0] - c[0]) + (c @ c) * (b[0] - a[0])) / d
    r = np.hypot(pts[:, 0] - ux, pts[:, 1] - uy)
    assert np.allclose(r, R, rtol=1e-9)


def test_boris_exb_drift():
    B = np.array([0.0, 0.0, 0.5])
    E = np.array([0.0, 200.0, 0.0])
    qm = 2 * QE / (40 * AMU)
    dt = 2e-8
    v = np.zeros(3)
    vs = []
    for _ in range(40000):
        v = O.boris(qm, E, B, dt, v)
        vs.append(v.copy())
    vd = np.cross(E, B) / (B @ B)
    mean = np.mean(vs, axis=0)
    assert mean[0] == pytest.approx(vd[0], rel=2e-2)
    assert abs(mean[1]) < 2e-2 * vd[0] and abs(mean[2]) < 1e-9


def _one_particle_run(rp, x, y, z, v, q):
    st = {"x": np.array([x]), "y": np.array([y]), "z": np.array([z]),
          "vx": np.array([v[0]]), "vy": np.array([v[1]]), "vz": np.array([v[2]]),
          "q": np.array([q])}
    return O.OracleRun(rp, st, deposit=False)


def test_mirror_magnetic_moment_invariant():
    # slow mirror, no hexapole: mu = M v_perp^2 / (2|B|) is an adiabatic invariant
    rp = I.RunParams(B_hex=0.0, flags=I.F_PUSH, dt=1e-9)
    p = O.make_params(rp)
    zm = 0.1848
    sp = math.sqrt(2 * 10 * QE / (40 * AMU))
    pitch = math.radians(60)
    r = _one_particle_run(rp, 0.002, 0.0, zm, [sp * math.sin(pitch), 0, sp * math.cos(pitch)], 8)
    mus, bs = [], []
    e0 = sp * sp
    for _ in range(600):
        r.step(100)
        Bv = O.bfield(p, r.x[0], r.y[0], r.z[0])
        b = np.linalg.norm(Bv)
        vv = np.array([r.vx[0], r.vy[0], r.vz[0]])
        vpar = vv @ Bv / b
        mus.append((vv @ vv - vpar * vpar) / b)
        bs.append(b)
        assert vv @ vv == pytest.approx(e0, rel=1e-9)   # pure magnetic field: energy kept
    mus = np.array(mus)
    # the ion bounces at the mirror point |B| = B_min / sin^2(pitch)
    assert max(bs) == pytest.approx(rp.B_min / math.sin(pitch) ** 2, rel=0.03)
    assert r.tally.lost[8] == 0 and r.tally.extracted[8] == 0
    assert (mus.max() - mus.min()) / mus.mean() < 0.03


def test_atoms_move_straight():
    rp = I.RunParams(flags=I.F_PUSH, dt=1e-9)
    r = _one_particle_run(rp, 0.001, 0.002, 0.1, [250.0, -120.0, 80.0], 0)
    r.step(1000)
    assert r.x[0] == pytest.approx(0.001 + 250.0 * 1e-6, rel=1e-12)
    assert r.y[0] == pytest.approx(0.002 - 120.0 * 1e-6, rel=1e-12)
    assert r.z[0] == pytest.approx(0.1 + 80.0 * 1e-6, rel=1e-12)
