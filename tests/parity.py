"""Lock-step and free-run comparison of the CUDA time step with the FP64 oracle.

Lock-step: before every step the oracle takes the GPU's FP32 state (as FP64),
advances it one step with the same counter-based random words, and the two
results are compared.  Integer outcomes (charge state, wall / aperture /
ionisation / charge-exchange events) must be identical for every particle
that the oracle did not flag as lying within rounding distance of a decision
surface (a cell face, a wall, the aperture edge, or an event threshold); for
flagged particles either outcome is admissible and only validity is checked.
Positions and velocities of unflagged particles agree to FP32 rounding.
"""
from __future__ import annotations

import numpy as np

from oracle import oracle as O

KEYS = ("x", "y", "z", "vx", "vy", "vz")
EV_MASK = 0x3F  # wall, extract, ionise, cx, coulomb, elastic


class Mismatch(AssertionError):
    pass


def coulomb_guard(rp, orc):
    """Particles whose Coulomb partners may differ: every ion in a cell (or a
    neighbouring cell) that holds an ion flagged near any decision surface."""
    dx, dy, dz = 2 * rp.R0 / rp.nx, 2 * rp.R0 / rp.ny, rp.L / rp.nz
    ix = np.clip(np.floor((orc.x + rp.R0) / dx).astype(np.int64), 0, rp.nx - 1)
    iy = np.clip(np.floor((orc.y + rp.R0) / dy).astype(np.int64), 0, rp.ny - 1)
    iz = np.clip(np.floor(orc.z / dz).astype(np.int64), 0, rp.nz - 1)
    bad = np.zeros((rp.nz + 2, rp.ny + 2, rp.nx + 2), dtype=bool)
    g = (orc.guard != 0) & (orc.q >= 1)
    for ox in (0, 1, 2):
        for oy in (0, 1, 2):
            for oz in (0, 1, 2):
                bad[iz[g] + oz, iy[g] + oy, ix[g] + ox] = True
    return bad[iz + 1, iy + 1, ix + 1] & (orc.q >= 1)


def compare_step(rp, g1, orc, pos_rel=1e-6, vel_rel=1e-5, v_floor=None, mask=O.G_SINGLE, probe=None, g0=None,
                 step=None):
    """Compare one GPU step (g1 = state after) with the oracle that took the same step.

    `mask` selects the guard bits that excuse a particle; with Coulomb
    collisions on, every ion near a flagged ion is excused as well.  With a
    probe oracle run, the pre-step GPU state g0 and the step index, a position
    mismatch is re-checked against the FP32 rounding of the handed-over start
    (handover_accepts)."""
    ok = (orc.guard & mask) == 0
    if rp.flags & O.F_COULOMB:
        ok &= (orc.guard == 0) & ~coulomb_guard(rp, orc)
    q_bad = (g1["q"] != orc.q) & ok
    ev_g = (g1["meta"] >> 8) & EV_MASK
    ev_bad = (ev_g != (orc.events & EV_MASK)) & ok
    # positions relative to the chamber size, velocities relative to |v| plus a floor
    same = ok & ~q_bad & ~ev_bad
    scale = {"x": rp.R0, "y": rp.R0, "z": rp.L}
    pos_bad = np.zeros_like(ok)
    for k in ("x", "y", "z"):
        pos_bad |= same & (np.abs(g1[k].astype(np.float64) - getattr(orc, k)) > pos_rel * scale[k])
    handover = 0
    if probe is not None and pos_bad.any():
        idx = np.nonzero(pos_bad)[0]
        acc = handover_accepts(rp, probe, g0, g1, orc, step, idx, pos_rel)
        pos_bad[idx[acc]] = False
        handover = int(acc.sum())
    vmag = np.sqrt(orc.vx ** 2 + orc.vy ** 2 + orc.vz ** 2)
    if v_floor is None:
        v_floor = np.sqrt(rp.T0_eV * 1.602176634e-19 / (rp.species.mass_amu * 1.66053906660e-27))
    vel_bad = np.zeros_like(ok)
    for k in ("vx", "vy", "vz"):
        vel_bad |= same & (np.abs(g1[k].astype(np.float64) - getattr(orc, k)) > vel_rel * (vmag + v_floor))
    bad = np.nonzero(q_bad | ev_bad | pos_bad | vel_bad)[0]
    detail = None
    if len(bad):
        i = int(bad[0])
        detail = {"i": i, "gpu": [float(g1[k][i]) for k in KEYS] + [int(g1["q"][i]), int(ev_g[i])],
                  "oracle": [float(getattr(orc, k)[i]) for k in KEYS] + [int(orc.q[i]), int(orc.events[i])],
                  "guard": int(orc.guard[i])}
    return {"handover": handover, "q": int(q_bad.sum()), "events": int(ev_bad.sum()), "pos": int(pos_bad.sum()),
            "vel": int(vel_bad.sum()), "guarded": int((~ok).sum()), "detail": detail}


def handover_accepts(rp, probe, g0, g1, orc, step, idx, pos_rel=1e-6):
    """The lock-step hands the oracle the FP32 export of the GPU's fixed-point
    positions, which is within one FP32 ulp of the true start.  A crossing at
    a grazing angle amplifies that rounding (by the ratio of the lateral to
    the normal displacement), so the re-emission point of a wall hit can
    differ by more than the position tolerance.  For the particles idx this
    re-runs the oracle step from the 8 corners of the one-ulp box around the
    exported start (same random words, same cell data) and accepts the GPU
    position when it lies within the spread of the corner outcomes that have
    the GPU's events, widened by the position tolerance.  Returns a boolean
    array over idx."""
    base = {k: g0[k].astype(np.float64) for k in KEYS}
    lo = {k: np.full(len(idx), np.inf) for k in ("x", "y", "z")}
    hi = {k: np.full(len(idx), -np.inf) for k in ("x", "y", "z")}
    ev_g = (g1["meta"][idx] >> 8) & EV_MASK
    status = np.where((g0["meta"] & (1 << 16)) != 0, 1, 0)
    for corner in range(8):
        st = {k: base[k].copy() for k in KEYS}
        st["q"] = g0["q"]
        for b, k in enumerate(("x", "y", "z")):
            toward = np.float32(np.inf if (corner >> b) & 1 else -np.inf)
            st[k][idx] = np.nextafter(g0[k][idx], toward, dtype=np.float32).astype(np.float64)
        probe.set_state(st)
        probe.status[:] = status
        probe.step_index = step
        probe.step(1)
        same = ((probe.events[idx] & EV_MASK) == ev_g) & (probe.q[idx] == g1["q"][idx])
        for k in ("x", "y", "z"):
            v = getattr(probe, k)[idx]
            lo[k] = np.where(same, np.minimum(lo[k], v), lo[k])
            hi[k] = np.where(same, np.maximum(hi[k], v), hi[k])
    scale = {"x": rp.R0, "y": rp.R0, "z": rp.L}
    ok = np.ones(len(idx), dtype=bool)
    for k in ("x", "y", "z"):
        v = g1[k][idx].astype(np.float64)
        ok &= (v >= lo[k] - pos_rel * scale[k]) & (v <= hi[k] + pos_rel * scale[k])
    return ok


def lockstep(run, rp, state0, steps, E=None, ne_cells=None, pos_rel=1e-6, vel_rel=1e-5, mask=O.G_SINGLE):
    """Drive the GPU run and the oracle step by step; returns totals and the oracle."""
    orc = O.OracleRun(rp, state0, E=E, ne_cells=ne_cells)
    probe = O.OracleRun(rp, state0, E=E, ne_cells=ne_cells, deposit=False)
    totals = {"q": 0, "events": 0, "pos": 0, "vel": 0, "guarded": 0, "handover": 0, "events_seen": 0}
    seen = np.zeros(16, dtype=np.int64)
    first_bad = None
    for s in range(steps):
        g0 = run.state()
        orc.set_state({k: g0[k] for k in KEYS + ("q",)})
        orc.status[:] = np.where((g0["meta"] & (1 << 16)) != 0, 1, 0)
        orc.step_index = s
        orc.step(1)
        run.step(1)
        g1 = run.state()
        r = compare_step(rp, g1, orc, pos_rel, vel_rel, mask=mask, probe=probe, g0=g0, step=s)
        for k in ("q", "events", "pos", "vel", "guarded", "handover"):
            totals[k] += r[k]
        if first_bad is None and (r["q"] or r["events"] or r["pos"] or r["vel"]):
            first_bad = {"step": s, "before": {k: float(g0[k][r["detail"]["i"]]) for k in KEYS},
                         **r["detail"]}
        for b in range(4):
            seen[b] += int(((orc.events >> b) & 1).sum())
    totals["events_seen"] = seen[:4].tolist()
    totals["first_bad"] = first_bad
    return totals, orc
