"""Lock-step comparison of the CUDA time step with the FP64 oracle.

Before every step the oracle takes the GPU's state (the FP32 export of its
fixed-point positions and its FP32 velocities, as FP64), advances it one step
with the same counter-based random words, and every particle's outcome is
compared: charge state and events exactly, positions to pos_rel of the
chamber size, velocities to vel_rel of |v| (plus a thermal floor).

A mismatch is accepted only where the oracle shows that the GPU took the
other side of a decision that lies within rounding distance of its surface,
and only if the GPU's whole outcome is the one the oracle gives on that other
side.  The oracle flags such decisions (guard bits): a cell face, a wall, the
aperture edge, a corner tie, an event threshold.  For each flag, probe runs of
the oracle step move the decision across its surface and nothing else by
more than rounding:

- positions (cell faces, walls, aperture edge, corner ties): the eight
  corners of the one-FP32-ulp box around the exported start, which brackets
  the GPU's exact fixed-point start;
- ionisation, double / triple ionisation and recombination thresholds: n_e
  of every cell scaled by 1 -/+ KAPPA (KAPPA is three times the oracle's
  threshold band, so each flagged word lands on both sides);
- charge-exchange and elastic thresholds: the background density n0 scaled
  by 1 -/+ KAPPA.

A flagged particle passes if its GPU outcome matches the probe of its flag.
With ion-ion collisions on, a flip changes the pairing of the cell it
happens in, so an ion without a flag passes a mismatch only if its cell (in
the main run or the probe) holds a flagged particle whose outcome that same
probe changed, and the ion matches that probe.  Everything else must match
the main oracle run.  A particle frozen at a wall (recycling off) is compared
at its position clamped into the box the fixed-point coordinates span.
"""
from __future__ import annotations


import numpy as np

from oracle import oracle as O

KEYS = ("x", "y", "z", "vx", "vy", "vz")
EV_MASK = 0x7F  # wall, extract, ionise, cx, coulomb, elastic, recombination
KAPPA = 3e-5    # relative probability shift of the threshold probes (the oracle's band is 1e-5)
G_POS = O.G_CELL | O.G_BOUNDARY | O.G_CELLREC
ST_FROZEN = 1 << 16


def _v_floor(rp):
    return np.sqrt(rp.T0_eV * 1.602176634e-19 / (rp.species.mass_amu * 1.66053906660e-27))


def mismatch(rp, g1, ref, pos_rel, vel_rel, v_floor=None):
    """Per-particle mismatch masks (q, events, position, velocity) of the GPU
    state g1 against an oracle run `ref` after the same step."""
    if v_floor is None:
        v_floor = _v_floor(rp)
    q_bad = g1["q"] != ref.q
    ev_g = (g1["meta"] >> 8) & EV_MASK
    ev_bad = ev_g != (ref.events & EV_MASK)
    frozen = (g1["meta"] & ST_FROZEN) != 0
    scale = {"x": rp.R0, "y": rp.R0, "z": rp.L}
    box = {"x": (-rp.R0, rp.R0), "y": (-rp.R0, rp.R0), "z": (0.0, rp.L)}
    pos_bad = np.zeros(len(q_bad), dtype=bool)
    for k in ("x", "y", "z"):
        r = getattr(ref, k)
        r = np.where(frozen, np.clip(r, *box[k]), r)
        pos_bad |= np.abs(g1[k].astype(np.float64) - r) > pos_rel * scale[k]
    vmag = np.sqrt(ref.vx ** 2 + ref.vy ** 2 + ref.vz ** 2)
    vel_bad = np.zeros(len(q_bad), dtype=bool)
    for k in ("vx", "vy", "vz"):
        vel_bad |= np.abs(g1[k].astype(np.float64) - getattr(ref, k)) > vel_rel * (vmag + v_floor)
    return q_bad, ev_bad, pos_bad, vel_bad


def as_state(run):
    """an oracle run's state in the GPU's export format (meta: events << 8,
    frozen status bit 16)"""
    meta = (run.events.astype(np.uint32) << 8) | (run.status.astype(np.uint32) << 16) | run.q.astype(np.uint32)
    return {"q": run.q, "meta": meta, **{k: getattr(run, k) for k in KEYS}}


def ngp(rp, run):
    dx, dy, dz = 2 * rp.R0 / rp.nx, 2 * rp.R0 / rp.ny, rp.L / rp.nz
    ix = np.clip(np.floor((run.x + rp.R0) / dx).astype(np.int64), 0, rp.nx - 1)
    iy = np.clip(np.floor((run.y + rp.R0) / dy).astype(np.int64), 0, rp.ny - 1)
    iz = np.clip(np.floor(run.z / dz).astype(np.int64), 0, rp.nz - 1)
    return (iz * rp.ny + iy) * rp.nx + ix


class Probes:
    """Oracle runs of one step from the handed-over state g0 with one kind of
    decision moved across its surface (see the module docstring); every other
    input (cell data, E grid, rates, parameters) is the main run's, `main`."""

    def __init__(self, rp, g0, step, main):
        self.rp, self.g0, self.step, self.main = rp, g0, step, main
        self.status = np.where((g0["meta"] & ST_FROZEN) != 0, 1, 0)
        self._runs = {}

    def _run(self, name):
        if name in self._runs:
            return self._runs[name]
        st = {k: self.g0[k].astype(np.float64) for k in KEYS}
        st["q"] = self.g0["q"]
        if name.startswith("corner"):
            c = int(name[6:])
            for b, k in enumerate(("x", "y", "z")):
                toward = np.float32(np.inf if (c >> b) & 1 else -np.inf)
                st[k] = np.nextafter(self.g0[k], toward, dtype=np.float32).astype(np.float64)
        m = self.main
        orc = O.OracleRun(self.rp, st, dt=m.p.dt, deposit=False)
        orc.E = m.E
        for k in ("ne", "zone", "dlx", "dly"):
            setattr(orc, k, np.ascontiguousarray(getattr(m, k).copy()))
        if name in ("ne+", "ne-"):
            orc.ne = np.ascontiguousarray(orc.ne * (1.0 + (KAPPA if name == "ne+" else -KAPPA)))
        if name in ("n0+", "n0-"):
            orc.p.n0_m3 *= 1.0 + (KAPPA if name == "n0+" else -KAPPA)
        orc.status[:] = self.status
        orc.step_index = self.step
        orc.step(1)
        self._runs[name] = orc
        return orc

    def kinds(self, guard_bits):
        """probe names and the guard bits each one targets"""
        out = []
        if guard_bits & G_POS:
            out += [(f"corner{c}", G_POS) for c in range(8)]
        if guard_bits & O.G_IONIZE:
            out += [("ne+", O.G_IONIZE), ("ne-", O.G_IONIZE)]
        if guard_bits & O.G_CX:
            out += [("n0+", O.G_CX), ("n0-", O.G_CX)]
        return out


def handover_spread(rp, probes, g1, idx, pos_rel):
    """Positions of particles idx whose events already match: the hand-over
    rounds the GPU's exact start to FP32, and a crossing at a grazing angle
    amplifies that rounding (by the ratio of the lateral to the normal
    displacement), so the re-emission point of a wall hit can move by more
    than the position tolerance.  Accept a GPU position inside the spread of
    the corner runs that have the GPU's events, widened by the tolerance."""
    ev_g = (g1["meta"][idx] >> 8) & EV_MASK
    lo = {k: np.full(len(idx), np.inf) for k in ("x", "y", "z")}
    hi = {k: np.full(len(idx), -np.inf) for k in ("x", "y", "z")}
    for c in range(8):
        pr = probes._run(f"corner{c}")
        same = ((pr.events[idx] & EV_MASK) == ev_g) & (pr.q[idx] == g1["q"][idx])
        for k in ("x", "y", "z"):
            v = getattr(pr, k)[idx]
            lo[k] = np.where(same, np.minimum(lo[k], v), lo[k])
            hi[k] = np.where(same, np.maximum(hi[k], v), hi[k])
    scale = {"x": rp.R0, "y": rp.R0, "z": rp.L}
    ok = np.ones(len(idx), dtype=bool)
    for k in ("x", "y", "z"):
        v = g1[k][idx].astype(np.float64)
        ok &= (v >= lo[k] - pos_rel * scale[k]) & (v <= hi[k] + pos_rel * scale[k])
    return ok


def compare_step(rp, g1, orc, pos_rel=1e-6, vel_rel=1e-5, probes=None, excuse=None):
    """Compare one GPU step (g1 = state after) with the oracle run that took the
    same step; mismatches are checked against the probes as described above.
    `excuse` (optional) marks particles a caller exempts for a stated reason;
    they are counted apart.  Returns counts of unexplained mismatches by kind,
    of mismatches the probes explain, of excused ones, of flagged particles,
    and the first unexplained one."""
    q_bad, ev_bad, pos_bad, vel_bad = mismatch(rp, g1, orc, pos_rel, vel_rel)
    res = {"guarded": int((orc.guard != 0).sum()), "accepted": 0, "handover": 0, "excused": 0}
    if excuse is not None:
        res["excused"] = int((excuse & (q_bad | ev_bad | pos_bad | vel_bad)).sum())
        q_bad, ev_bad, pos_bad, vel_bad = (a & ~excuse for a in (q_bad, ev_bad, pos_bad, vel_bad))
    bad = q_bad | ev_bad | pos_bad | vel_bad
    guard = orc.guard.astype(np.int64)
    if bad.any() and probes is not None:
        accepted = np.zeros(len(bad), dtype=bool)
        coulomb = (rp.flags & O.F_COULOMB) != 0
        # position-only mismatches: the hand-over spread
        pos_only = np.nonzero(bad & pos_bad & ~q_bad & ~ev_bad & ~vel_bad)[0]
        if len(pos_only):
            acc = handover_spread(rp, probes, g1, pos_only, pos_rel)
            accepted[pos_only[acc]] = True
            res["handover"] = int(acc.sum())
        rest = bad & ~accepted
        if rest.any():
            cell_main = ngp(rp, orc) if coulomb else None
            for name, target in probes.kinds(int(np.bitwise_or.reduce(guard[guard != 0])) if res["guarded"]
                                               else 0):
                if not rest.any():
                    break
                pr = probes._run(name)
                pq, pe, pp, pv = mismatch(rp, g1, pr, pos_rel, vel_rel)
                match = ~(pq | pe | pp | pv)
                own = (guard & target) != 0
                ok = rest & match & own
                if coulomb:
                    # flagged particles whose outcome this probe changed, and
                    # the cells they collide in (main run and probe)
                    dq, de, dp, dv = mismatch(rp, as_state(pr), orc, pos_rel, vel_rel)
                    flipped = own & (dq | de | dp | dv)
                    if flipped.any():
                        touched = np.union1d(cell_main[flipped], ngp(rp, pr)[flipped])
                        ion = g1["q"] >= 1
                        in_cell = np.isin(cell_main, touched) | np.isin(ngp(rp, pr), touched)
                        ok |= rest & match & ion & in_cell
                accepted |= ok
                rest &= ~ok
        res["accepted"] = int(accepted.sum())
        q_bad &= ~accepted
        ev_bad &= ~accepted
        pos_bad &= ~accepted
        vel_bad &= ~accepted
    first = np.nonzero(q_bad | ev_bad | pos_bad | vel_bad)[0]
    detail = None
    if len(first):
        i = int(first[0])
        ev_g = (g1["meta"] >> 8) & EV_MASK
        detail = {"i": i, "gpu": [float(g1[k][i]) for k in KEYS] + [int(g1["q"][i]), int(ev_g[i])],
                  "oracle": [float(getattr(orc, k)[i]) for k in KEYS] + [int(orc.q[i]), int(orc.events[i])],
                  "guard": int(orc.guard[i])}
    res.update({"q": int(q_bad.sum()), "events": int(ev_bad.sum()), "pos": int(pos_bad.sum()),
                "vel": int(vel_bad.sum()), "detail": detail})
    return res


def lockstep(run, rp, state0, steps, E=None, ne_cells=None, pos_rel=1e-6, vel_rel=1e-5):
    """Drive the GPU run and the oracle step by step; returns the totals
    (unexplained mismatches by kind, explained ones, flagged particle-steps
    and their fraction, events seen, the first unexplained mismatch) and the
    main oracle run."""
    orc = O.OracleRun(rp, state0, E=E, ne_cells=ne_cells)
    totals = {"q": 0, "events": 0, "pos": 0, "vel": 0, "guarded": 0, "accepted": 0, "handover": 0,
              "events_seen": 0}
    seen = np.zeros(16, dtype=np.int64)
    first_bad = None
    n = len(state0["x"])
    for s in range(steps):
        g0 = run.state()
        orc.set_state({k: g0[k] for k in KEYS + ("q",)})
        orc.status[:] = np.where((g0["meta"] & ST_FROZEN) != 0, 1, 0)
        orc.step_index = s
        orc.step(1)
        run.step(1)
        g1 = run.state()
        r = compare_step(rp, g1, orc, pos_rel, vel_rel, probes=Probes(rp, g0, s, orc))
        for k in ("q", "events", "pos", "vel", "guarded", "accepted", "handover"):
            totals[k] += r[k]
        if first_bad is None and (r["q"] or r["events"] or r["pos"] or r["vel"]):
            first_bad = {"step": s, "before": {k: float(g0[k][r["detail"]["i"]]) for k in KEYS},
                         **r["detail"]}
        for b in range(7):
            seen[b] += int(((orc.events >> b) & 1).sum())
    totals["events_seen"] = seen[:4].tolist()
    totals["events_seen_all"] = seen[:7].tolist()
    totals["guarded_frac"] = totals["guarded"] / max(1, n * steps)
    totals["accepted_frac"] = totals["accepted"] / max(1, n * steps)
    totals["first_bad"] = first_bad
    return totals, orc
