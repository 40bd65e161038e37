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
EV_MASK = 0xF  # wall, extract, ionise, cx


class Mismatch(AssertionError):
    pass


def compare_step(rp, g1, orc, pos_rel=1e-6, vel_rel=1e-5, v_floor=None):
    """Compare one GPU step (g1 = state after) with the oracle that took the same step."""
    ok = orc.guard == 0
    q_bad = (g1["q"] != orc.q) & ok
    ev_g = (g1["meta"] >> 8) & EV_MASK
    ev_bad = (ev_g != (orc.events & EV_MASK)) & ok
    # positions relative to the chamber size, velocities relative to |v| plus a floor
    same = ok & ~q_bad & ~ev_bad
    scale = {"x": rp.R0, "y": rp.R0, "z": rp.L}
    pos_bad = np.zeros_like(ok)
    for k in ("x", "y", "z"):
        pos_bad |= same & (np.abs(g1[k].astype(np.float64) - getattr(orc, k)) > pos_rel * scale[k])
    vmag = np.sqrt(orc.vx ** 2 + orc.vy ** 2 + orc.vz ** 2)
    if v_floor is None:
        v_floor = np.sqrt(rp.T0_eV * 1.602176634e-19 / (rp.species.mass_amu * 1.66053906660e-27))
    vel_bad = np.zeros_like(ok)
    for k in ("vx", "vy", "vz"):
        vel_bad |= same & (np.abs(g1[k].astype(np.float64) - getattr(orc, k)) > vel_rel * (vmag + v_floor))
    return {"q": int(q_bad.sum()), "events": int(ev_bad.sum()), "pos": int(pos_bad.sum()),
            "vel": int(vel_bad.sum()), "guarded": int((~ok).sum()),
            "bad_idx": np.nonzero(q_bad | ev_bad | pos_bad | vel_bad)[0][:10]}


def lockstep(run, rp, state0, steps, E=None, ne_cells=None, pos_rel=1e-6, vel_rel=1e-5):
    """Drive the GPU run and the oracle step by step; returns totals and the oracle."""
    orc = O.OracleRun(rp, state0, E=E, ne_cells=ne_cells)
    totals = {"q": 0, "events": 0, "pos": 0, "vel": 0, "guarded": 0, "events_seen": 0}
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
        r = compare_step(rp, g1, orc, pos_rel, vel_rel)
        for k in ("q", "events", "pos", "vel", "guarded"):
            totals[k] += r[k]
        if first_bad is None and (r["q"] or r["events"] or r["pos"] or r["vel"]):
            first_bad = (s, r)
        for b in range(4):
            seen[b] += int(((orc.events >> b) & 1).sum())
    totals["events_seen"] = seen[:4].tolist()
    totals["first_bad"] = first_bad
    return totals, orc
