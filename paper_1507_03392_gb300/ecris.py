"""Python binding of the ECRIS C ABI (include/ecris.h).

Argument marshalling only: every step of the time step runs in the CUDA
library libecris.so, which this module loads from the package directory.  If
the library is missing, importing this module raises; there is no fallback.

The functions `ecris_create`, `ecris_destroy`, `ecris_last_error`,
`ecris_init_fields`, `ecris_load_ions`, `ecris_step`, `ecris_diag` and
`ecris_get_state` carry the C names and signatures.  `Run` wraps them for one
run described by `inputs.RunParams`, taking numpy arrays (host) or torch CUDA
tensors (device) for the particle state.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libecris.so")

ECRIS_OK, ECRIS_EINVAL, ECRIS_ENOMEM, ECRIS_ECUDA, ECRIS_ETIMEOUT, ECRIS_ESTATE = range(6)
STATUS_NAMES = {0: "ECRIS_OK", 1: "ECRIS_EINVAL", 2: "ECRIS_ENOMEM", 3: "ECRIS_ECUDA",
                4: "ECRIS_ETIMEOUT", 5: "ECRIS_ESTATE"}
EV_WALL, EV_EXTRACT, EV_IONIZE, EV_CX, EV_COULOMB = (1 << 8, 1 << 9, 1 << 10, 1 << 11, 1 << 12)
ST_FROZEN = 1 << 16


class EcrisError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class Geometry(ctypes.Structure):
    _fields_ = [("R0", ctypes.c_double), ("L", ctypes.c_double), ("r_ap", ctypes.c_double),
                ("inlet", ctypes.c_double * 3)]


class BField(ctypes.Structure):
    _fields_ = [("B_inj", ctypes.c_double), ("B_min", ctypes.c_double), ("B_ext", ctypes.c_double),
                ("B_hex", ctypes.c_double), ("B_ecr", ctypes.c_double),
                ("n_axial", ctypes.c_int32), ("B_axial", ctypes.c_void_p)]


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("E", ctypes.c_void_p), ("ne_in_cm3", ctypes.c_double),
                ("ne_in_cells", ctypes.c_void_p), ("ne_out_cm3", ctypes.c_double),
                ("Te_warm_eV", ctypes.c_double), ("Te_cold_eV", ctypes.c_double)]


class Species(ctypes.Structure):
    _fields_ = [("mass_amu", ctypes.c_double), ("qmax", ctypes.c_int32),
                ("ip_eV", ctypes.c_void_p), ("n_outer", ctypes.c_void_p)]


class Mcc(ctypes.Structure):
    _fields_ = [("n0_cm3", ctypes.c_double), ("T0_eV", ctypes.c_double),
                ("sigma1_cm2", ctypes.c_double), ("E_cx_eV", ctypes.c_double),
                ("lnL_ii", ctypes.c_double), ("lnL_ei", ctypes.c_double),
                ("ei_charge_power", ctypes.c_int32), ("flags", ctypes.c_uint32),
                ("T_refl_eV", ctypes.c_double), ("sigma_el1_cm2", ctypes.c_double), ("k2_factor", ctypes.c_double),
                ("k3_factor", ctypes.c_double)]


class DiagOut(ctypes.Structure):
    _fields_ = [("qmax", ctypes.c_int32), ("steps", ctypes.c_uint64), ("time_s", ctypes.c_double),
                ("extracted", ctypes.c_void_p), ("lost", ctypes.c_void_p),
                ("alive_by_q", ctypes.c_void_p), ("current_A", ctypes.c_void_p),
                ("ke_lost_eV", ctypes.c_double), ("power_W", ctypes.c_double),
                ("coulomb_collisions", ctypes.c_int64),
                ("cell_count", ctypes.c_void_p), ("cell_charge", ctypes.c_void_p)]


class Tuning(ctypes.Structure):
    _fields_ = [("sort_every", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("threads", ctypes.c_int32), ("particles_per_thread", ctypes.c_int32),
                ("stages", ctypes.c_int32), ("reserved", ctypes.c_int32 * 3)]


class Request(ctypes.Structure):
    _fields_ = [("geo", Geometry), ("bf", BField), ("grid", Grid), ("sp", Species), ("mcc", Mcc),
                ("n", ctypes.c_size_t), ("xyzv", ctypes.c_void_p * 6), ("q", ctypes.c_void_p),
                ("weight", ctypes.c_double), ("seed", ctypes.c_uint64), ("dt", ctypes.c_double),
                ("window_steps", ctypes.c_uint32), ("rel_tol", ctypes.c_double),
                ("min_events", ctypes.c_int64), ("max_steps", ctypes.c_uint32), ("ne_windows", ctypes.c_uint32)]


class Result(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("converged", ctypes.c_int32), ("steps", ctypes.c_uint64),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double),
                ("qmax", ctypes.c_int32), ("extracted", ctypes.c_int64 * 64), ("lost", ctypes.c_int64 * 64),
                ("current_A", ctypes.c_double * 64), ("power_W", ctypes.c_double),
                ("ke_lost_eV", ctypes.c_double), ("error", ctypes.c_char * 128),
                ("flow_per_s", ctypes.c_double), ("power_window_W", ctypes.c_double)]


REQ_QUEUED, REQ_RUNNING, REQ_DONE, REQ_FAILED = 0, 1, 2, 3
CALIB_HISTORY = 32   # ECRIS_CALIB_HISTORY


class CalibRequest(ctypes.Structure):
    _fields_ = [("base", Request), ("flow_target", ctypes.c_double), ("power_target_W", ctypes.c_double),
                ("tol", ctypes.c_double), ("max_iter", ctypes.c_int32)]


class CalibResult(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("met", ctypes.c_int32), ("iterations", ctypes.c_int32),
                ("weight", ctypes.c_double * CALIB_HISTORY), ("Te_warm_eV", ctypes.c_double * CALIB_HISTORY),
                ("flow_per_s", ctypes.c_double * CALIB_HISTORY), ("power_W", ctypes.c_double * CALIB_HISTORY),
                ("steps", ctypes.c_uint64 * CALIB_HISTORY), ("error", ctypes.c_char * 128)]


MAX_SCREENS = 4   # ECRIS_MAX_SCREENS


class ProbeSpec(ctypes.Structure):
    _fields_ = [("ncells", ctypes.c_size_t), ("cells", ctypes.c_void_p), ("nscreens", ctypes.c_int32),
                ("z_lo", ctypes.c_double * MAX_SCREENS), ("z_hi", ctypes.c_double * MAX_SCREENS),
                ("pixels", ctypes.c_int32)]


class Profile(ctypes.Structure):
    _fields_ = [("step_launches", ctypes.c_int64), ("step_ms", ctypes.c_double),
                ("coulomb_launches", ctypes.c_int64), ("coulomb_ms", ctypes.c_double),
                ("other_launches", ctypes.c_int64), ("other_ms", ctypes.c_double)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"CUDA library {LIB_PATH} is not built; run "
                          "`python -c 'import __graft_entry__ as g; g.build()'` first")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    st = ctypes.c_int
    lib.ecris_create.argtypes = [ctypes.POINTER(P), ctypes.c_int, P]
    lib.ecris_create.restype = st
    lib.ecris_destroy.argtypes = [P]
    lib.ecris_destroy.restype = None
    lib.ecris_last_error.argtypes = [P]
    lib.ecris_last_error.restype = ctypes.c_char_p
    lib.ecris_init_fields.argtypes = [P, ctypes.POINTER(Geometry), ctypes.POINTER(BField),
                                      ctypes.POINTER(Grid), ctypes.POINTER(Species), ctypes.POINTER(Mcc)]
    lib.ecris_init_fields.restype = st
    lib.ecris_load_ions.argtypes = [P, ctypes.c_size_t, ctypes.POINTER(P), P, ctypes.c_double,
                                    ctypes.c_uint64, ctypes.c_int]
    lib.ecris_load_ions.restype = st
    lib.ecris_step.argtypes = [P, ctypes.c_uint32, ctypes.c_double]
    lib.ecris_step.restype = st
    lib.ecris_diag.argtypes = [P, ctypes.POINTER(DiagOut)]
    lib.ecris_diag.restype = st
    lib.ecris_get_state.argtypes = [P, ctypes.POINTER(P), P, ctypes.c_int]
    lib.ecris_get_state.restype = st
    lib.ecris_update_ne.argtypes = [P]
    lib.ecris_update_ne.restype = st
    lib.ecris_get_cells.argtypes = [P, P, P, P]
    lib.ecris_get_cells.restype = st
    lib.ecris_get_fptd.argtypes = [P, P, P]
    lib.ecris_get_fptd.restype = st
    lib.ecris_get_extraction_radius.argtypes = [P, P]
    lib.ecris_get_extraction_radius.restype = st
    lib.ecris_set_probes.argtypes = [P, ctypes.POINTER(ProbeSpec)]
    lib.ecris_set_probes.restype = st
    lib.ecris_probe_sample.argtypes = [P]
    lib.ecris_probe_sample.restype = st
    lib.ecris_get_probes.argtypes = [P, P, P, P]
    lib.ecris_get_probes.restype = st
    lib.ecris_set_profiling.argtypes = [P, ctypes.c_int]
    lib.ecris_set_profiling.restype = st
    lib.ecris_get_profile.argtypes = [P, ctypes.POINTER(Profile)]
    lib.ecris_get_profile.restype = st
    lib.ecris_coulomb_collide_noalloc.argtypes = [ctypes.c_size_t, P, P, P, P, P, P, ctypes.c_uint32,
                                                  ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                                  ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                                  ctypes.c_uint32, P, ctypes.POINTER(ctypes.c_int64)]
    lib.ecris_coulomb_collide_noalloc.restype = st
    lib.ecris_set_tuning.argtypes = [P, ctypes.POINTER(Tuning)]
    lib.ecris_set_tuning.restype = st
    lib.ecris_batch_create.argtypes = [ctypes.POINTER(P), ctypes.c_int, P, ctypes.c_size_t]
    lib.ecris_batch_create.restype = st
    lib.ecris_batch_destroy.argtypes = [P]
    lib.ecris_batch_destroy.restype = None
    lib.ecris_batch_last_error.argtypes = [P]
    lib.ecris_batch_last_error.restype = ctypes.c_char_p
    lib.ecris_run_bytes.argtypes = [ctypes.c_size_t, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int]
    lib.ecris_run_bytes.restype = ctypes.c_size_t
    lib.ecris_batch_add_run.argtypes = [P, ctypes.POINTER(Geometry), ctypes.POINTER(BField), ctypes.POINTER(Grid),
                                        ctypes.POINTER(Species), ctypes.POINTER(Mcc), ctypes.c_size_t,
                                        ctypes.POINTER(P), P, ctypes.c_double, ctypes.c_uint64, ctypes.c_double,
                                        ctypes.c_int, ctypes.POINTER(ctypes.c_int32)]
    lib.ecris_batch_add_run.restype = st
    lib.ecris_batch_remove_run.argtypes = [P, ctypes.c_int32]
    lib.ecris_batch_remove_run.restype = st
    lib.ecris_batch_step.argtypes = [P, ctypes.c_uint32]
    lib.ecris_batch_step.restype = st
    lib.ecris_batch_diag.argtypes = [P, ctypes.c_int32, ctypes.POINTER(DiagOut)]
    lib.ecris_batch_diag.restype = st
    lib.ecris_batch_get_state.argtypes = [P, ctypes.c_int32, ctypes.POINTER(P), P, ctypes.c_int]
    lib.ecris_batch_get_state.restype = st
    lib.ecris_batch_update_ne.argtypes = [P, ctypes.c_int32]
    lib.ecris_batch_update_ne.restype = st
    lib.ecris_batch_get_cells.argtypes = [P, ctypes.c_int32, P, P, P]
    lib.ecris_batch_get_cells.restype = st
    lib.ecris_batch_get_fptd.argtypes = [P, ctypes.c_int32, P, P]
    lib.ecris_batch_get_fptd.restype = st
    lib.ecris_batch_get_extraction_radius.argtypes = [P, ctypes.c_int32, P]
    lib.ecris_batch_get_extraction_radius.restype = st
    lib.ecris_batch_set_probes.argtypes = [P, ctypes.c_int32, ctypes.POINTER(ProbeSpec)]
    lib.ecris_batch_set_probes.restype = st
    lib.ecris_batch_probe_sample.argtypes = [P, ctypes.c_int32]
    lib.ecris_batch_probe_sample.restype = st
    lib.ecris_batch_get_probes.argtypes = [P, ctypes.c_int32, P, P, P]
    lib.ecris_batch_get_probes.restype = st
    lib.ecris_batch_memory.argtypes = [P, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)]
    lib.ecris_batch_memory.restype = st
    lib.ecris_batch_autotune.argtypes = [P, ctypes.c_uint32, ctypes.POINTER(Tuning)]
    lib.ecris_batch_autotune.restype = st
    lib.ecris_batch_set_tuning.argtypes = [P, ctypes.POINTER(Tuning)]
    lib.ecris_batch_set_tuning.restype = st
    lib.ecris_batch_set_profiling.argtypes = [P, ctypes.c_int]
    lib.ecris_batch_set_profiling.restype = st
    lib.ecris_batch_get_profile.argtypes = [P, ctypes.POINTER(Profile)]
    lib.ecris_batch_get_profile.restype = st
    lib.ecris_server_create.argtypes = [ctypes.POINTER(P), ctypes.c_int, ctypes.c_size_t, ctypes.c_uint32,
                                        ctypes.c_uint32]
    lib.ecris_server_create.restype = st
    lib.ecris_server_destroy.argtypes = [P]
    lib.ecris_server_destroy.restype = None
    lib.ecris_server_last_error.argtypes = [P]
    lib.ecris_server_last_error.restype = ctypes.c_char_p
    lib.ecris_server_submit.argtypes = [P, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_int64)]
    lib.ecris_server_submit.restype = st
    lib.ecris_server_poll.argtypes = [P, ctypes.c_int64, ctypes.POINTER(Result)]
    lib.ecris_server_poll.restype = st
    d = ctypes.POINTER(ctypes.c_double)
    i64 = ctypes.POINTER(ctypes.c_int64)
    lib.ecris_server_stats.argtypes = [P, d, i64, i64, i64, d]
    lib.ecris_server_stats.restype = st
    lib.ecris_server_tunings.argtypes = [P, ctypes.POINTER(ctypes.c_int64)]
    lib.ecris_server_tunings.restype = st
    lib.ecris_server_calibrate.argtypes = [P, ctypes.POINTER(CalibRequest), i64]
    lib.ecris_server_calibrate.restype = st
    lib.ecris_server_calib_poll.argtypes = [P, ctypes.c_int64, ctypes.POINTER(CalibResult)]
    lib.ecris_server_calib_poll.restype = st
    return lib


LIB = _load()

# ---- the C entry points under their own names --------------------------------
ecris_create = LIB.ecris_create
ecris_destroy = LIB.ecris_destroy
ecris_last_error = LIB.ecris_last_error
ecris_init_fields = LIB.ecris_init_fields
ecris_load_ions = LIB.ecris_load_ions
ecris_step = LIB.ecris_step
ecris_diag = LIB.ecris_diag
ecris_get_state = LIB.ecris_get_state
ecris_update_ne = LIB.ecris_update_ne
ecris_get_cells = LIB.ecris_get_cells
ecris_get_fptd = LIB.ecris_get_fptd
ecris_get_extraction_radius = LIB.ecris_get_extraction_radius
ecris_set_probes = LIB.ecris_set_probes
ecris_probe_sample = LIB.ecris_probe_sample
ecris_get_probes = LIB.ecris_get_probes
ecris_set_profiling = LIB.ecris_set_profiling
ecris_get_profile = LIB.ecris_get_profile
ecris_coulomb_collide_noalloc = LIB.ecris_coulomb_collide_noalloc
ecris_set_tuning = LIB.ecris_set_tuning
ecris_batch_create = LIB.ecris_batch_create
ecris_batch_destroy = LIB.ecris_batch_destroy
ecris_batch_last_error = LIB.ecris_batch_last_error
ecris_run_bytes = LIB.ecris_run_bytes
ecris_batch_add_run = LIB.ecris_batch_add_run
ecris_batch_remove_run = LIB.ecris_batch_remove_run
ecris_batch_step = LIB.ecris_batch_step
ecris_batch_diag = LIB.ecris_batch_diag
ecris_batch_get_state = LIB.ecris_batch_get_state
ecris_batch_update_ne = LIB.ecris_batch_update_ne
ecris_batch_get_cells = LIB.ecris_batch_get_cells
ecris_batch_get_fptd = LIB.ecris_batch_get_fptd
ecris_batch_get_extraction_radius = LIB.ecris_batch_get_extraction_radius
ecris_batch_set_probes = LIB.ecris_batch_set_probes
ecris_batch_probe_sample = LIB.ecris_batch_probe_sample
ecris_batch_get_probes = LIB.ecris_batch_get_probes
ecris_batch_memory = LIB.ecris_batch_memory
ecris_batch_autotune = LIB.ecris_batch_autotune
ecris_batch_set_tuning = LIB.ecris_batch_set_tuning
ecris_batch_set_profiling = LIB.ecris_batch_set_profiling
ecris_batch_get_profile = LIB.ecris_batch_get_profile
ecris_server_create = LIB.ecris_server_create
ecris_server_destroy = LIB.ecris_server_destroy
ecris_server_last_error = LIB.ecris_server_last_error
ecris_server_submit = LIB.ecris_server_submit
ecris_server_poll = LIB.ecris_server_poll
ecris_server_stats = LIB.ecris_server_stats
ecris_server_tunings = LIB.ecris_server_tunings
ecris_server_calibrate = LIB.ecris_server_calibrate
ecris_server_calib_poll = LIB.ecris_server_calib_poll


def check(ctx, status):
    if status != ECRIS_OK:
        msg = ecris_last_error(ctx)
        raise EcrisError(status, msg.decode() if msg else "")
    return status


def _ptr(a):
    """Address of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


def _is_device(a):
    return not isinstance(a, np.ndarray) and getattr(a, "is_cuda", False)


def current_stream_handle():
    """cudaStream_t of torch's current stream on the current device."""
    import torch
    return torch.cuda.current_stream().cuda_stream


def field_structs(rp, E=None, ne_cells=None):
    """ecris_init_fields arguments for an inputs.RunParams (plus the arrays they point to)."""
    geo = Geometry(rp.R0, rp.L, rp.r_ap, (ctypes.c_double * 3)(*rp.inlet))
    bax = None if rp.B_axial is None else np.ascontiguousarray(rp.B_axial, dtype=np.float64)
    bf = BField(rp.B_inj, rp.B_min, rp.B_ext, rp.B_hex, rp.B_ecr, 0 if bax is None else len(bax), _ptr(bax))
    Eh = None if E is None else np.ascontiguousarray(E, dtype=np.float32).reshape(-1)
    nh = None if ne_cells is None else np.ascontiguousarray(ne_cells, dtype=np.float32)
    grid = Grid(rp.nx, rp.ny, rp.nz, _ptr(Eh), rp.ne_in_cm3, _ptr(nh), rp.ne_out_cm3,
                rp.Te_warm_eV, rp.Te_cold_eV)
    ip, nout = rp.species.ladder()
    ip = np.ascontiguousarray(ip, np.float64)
    nout = np.ascontiguousarray(nout, np.int32)
    sp = Species(rp.species.mass_amu, rp.species.qmax, _ptr(ip), _ptr(nout))
    mcc = Mcc(rp.n0_cm3, rp.T0_eV, rp.sigma1_cm2, rp.E_cx_eV, rp.lnL_ii, rp.lnL_ei,
              rp.ei_charge_power, rp.flags, rp.T_refl_eV, rp.sigma_el1_cm2, rp.k2_factor, rp.k3_factor)
    return geo, bf, grid, sp, mcc, (Eh, nh, ip, nout, bax)


def _state_arrays(state):
    arrs = [state[k] for k in ("x", "y", "z", "vx", "vy", "vz")]
    q = state["q"]
    dev = _is_device(arrs[0])
    if not dev:
        arrs = [np.ascontiguousarray(a, dtype=np.float32) for a in arrs]
        q = np.ascontiguousarray(q, dtype=np.uint8)
    return arrs, q, dev


def _diag(qmax, ncells, fn, grids=False):
    q1 = qmax + 1
    ext = np.zeros(q1, np.int64)
    lost = np.zeros(q1, np.int64)
    alive = np.zeros(q1, np.int64)
    cur = np.zeros(q1, np.float64)
    cc = np.zeros(ncells, np.uint64) if grids else None
    cq = np.zeros(ncells, np.uint64) if grids else None
    out = DiagOut(0, 0, 0.0, _ptr(ext), _ptr(lost), _ptr(alive), _ptr(cur), 0.0, 0.0, 0, _ptr(cc), _ptr(cq))
    fn(ctypes.byref(out))
    d = {"steps": out.steps, "time_s": out.time_s, "extracted": ext, "lost": lost,
         "alive_by_q": alive, "current_A": cur, "ke_lost_eV": out.ke_lost_eV,
         "power_W": out.power_W, "coulomb_collisions": out.coulomb_collisions}
    if grids:
        d["cell_count"], d["cell_charge"] = cc, cq
    return d


def _state(n, fn):
    arrs = [np.zeros(n, np.float32) for _ in range(6)]
    meta = np.zeros(n, np.uint32)
    ptrs = (ctypes.c_void_p * 6)(*[_ptr(a) for a in arrs])
    fn(ptrs, _ptr(meta))
    d = dict(zip(("x", "y", "z", "vx", "vy", "vz"), arrs))
    d["meta"] = meta
    d["q"] = (meta & 0xFF).astype(np.int32)
    return d


class Batch:
    """Many runs stepped together on one GPU (ecris_batch_*)."""

    def __init__(self, device=0, stream=None, hbm_budget=0):
        self.b = ctypes.c_void_p()
        st = ecris_batch_create(ctypes.byref(self.b), int(device), stream, int(hbm_budget))
        if st != ECRIS_OK:
            raise EcrisError(st, ecris_batch_last_error(None).decode())
        self.runs = {}

    def _check(self, st):
        if st != ECRIS_OK:
            raise EcrisError(st, ecris_batch_last_error(self.b).decode())

    def close(self):
        if self.b:
            ecris_batch_destroy(self.b)
            self.b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add(self, rp, state, E=None, ne_cells=None, weight=None, seed=None, dt=None):
        """Add a run; returns its handle."""
        f = field_structs(rp, E, ne_cells)
        arrs, q, dev = _state_arrays(state)
        ptrs = (ctypes.c_void_p * 6)(*[_ptr(a) for a in arrs])
        h = ctypes.c_int32(-1)
        self._check(ecris_batch_add_run(self.b, *[ctypes.byref(x) for x in f[:5]], len(arrs[0]), ptrs, _ptr(q),
                                        rp.weight if weight is None else weight,
                                        rp.seed if seed is None else seed, rp.dt if dt is None else dt,
                                        1 if dev else 0, ctypes.byref(h)))
        self.runs[h.value] = (rp, len(arrs[0]))
        return h.value

    def remove(self, h):
        self._check(ecris_batch_remove_run(self.b, int(h)))
        self.runs.pop(h, None)

    def step(self, nsteps=1):
        self._check(ecris_batch_step(self.b, int(nsteps)))

    def diag(self, h, grids=False):
        rp, n = self.runs[h]
        return _diag(rp.species.qmax, rp.ncells, lambda o: self._check(ecris_batch_diag(self.b, int(h), o)), grids)

    def state(self, h):
        rp, n = self.runs[h]
        return _state(n, lambda p, m: self._check(ecris_batch_get_state(self.b, int(h), p, m, 0)))

    def update_ne(self, h):
        self._check(ecris_batch_update_ne(self.b, int(h)))

    def extraction_radius(self, h):
        rp, _ = self.runs[h]
        return _radius(rp.species.qmax, lambda a: self._check(ecris_batch_get_extraction_radius(self.b, int(h), a)))

    def set_probes(self, h, cells=None, screens=(), pixels=256):
        sp, keep = _probe_spec(cells, screens, pixels)
        self._check(ecris_batch_set_probes(self.b, int(h), ctypes.byref(sp)))
        self._probe_shape = getattr(self, "_probe_shape", {})
        self._probe_shape[h] = (len(keep), len(screens), int(pixels))

    def probe_sample(self, h):
        self._check(ecris_batch_probe_sample(self.b, int(h)))

    def probes(self, h):
        rp, _ = self.runs[h]
        nc, ns, px = self._probe_shape[h]
        return _probes(rp.species.qmax, nc, ns, px,
                       lambda a, b, c: self._check(ecris_batch_get_probes(self.b, int(h), a, b, c)))

    def fptd(self, h):
        rp, _ = self.runs[h]
        return _fptd(rp.species.qmax, lambda a, b: self._check(ecris_batch_get_fptd(self.b, int(h), a, b)))

    def cells(self, h):
        rp, _ = self.runs[h]
        return _cells(rp.ncells, lambda a, b, c: self._check(ecris_batch_get_cells(self.b, int(h), a, b, c)))

    def memory(self):
        u, b = ctypes.c_size_t(0), ctypes.c_size_t(0)
        self._check(ecris_batch_memory(self.b, ctypes.byref(u), ctypes.byref(b)))
        return u.value, b.value

    def autotune(self, trial_steps=4):
        """choose the launch shape, blocks per SM and sort cadence by timing
        (the runs' state is restored after the trials)"""
        t = Tuning()
        self._check(ecris_batch_autotune(self.b, int(trial_steps), ctypes.byref(t)))
        return {"sort_every": t.sort_every, "blocks_per_sm": t.blocks_per_sm, "threads": t.threads,
                "particles_per_thread": t.particles_per_thread, "stages": t.stages}

    def set_tuning(self, sort_every=32, blocks_per_sm=0, threads=0, particles_per_thread=0, stages=0):
        t = Tuning()
        t.sort_every, t.blocks_per_sm = int(sort_every), int(blocks_per_sm)
        t.threads, t.particles_per_thread, t.stages = int(threads), int(particles_per_thread), int(stages)
        self._check(ecris_batch_set_tuning(self.b, ctypes.byref(t)))

    def set_profiling(self, on=True):
        self._check(ecris_batch_set_profiling(self.b, 1 if on else 0))

    def profile(self):
        p = Profile()
        self._check(ecris_batch_get_profile(self.b, ctypes.byref(p)))
        return {f: getattr(p, f) for f, _ in Profile._fields_}


class Server:
    """The served form (ecris_server_*): submit runs, poll their results."""

    def __init__(self, device=0, hbm_budget=0, steps_per_tick=32, max_active=0):
        self.s = ctypes.c_void_p()
        st = ecris_server_create(ctypes.byref(self.s), int(device), int(hbm_budget), int(steps_per_tick),
                                 int(max_active))
        if st != ECRIS_OK:
            raise EcrisError(st, "server_create failed")

    def close(self):
        if self.s:
            ecris_server_destroy(self.s)
            self.s = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _request(self, rp, state, E, ne_cells, window_steps, rel_tol, min_events, max_steps, weight, seed, dt,
                 ne_windows=0):
        """ecris_request for rp and state, with the arrays it points to."""
        f = field_structs(rp, E, ne_cells)
        arrs, q, dev = _state_arrays(state)
        if dev:
            raise ValueError("the server copies host arrays; pass numpy arrays")
        r = Request()
        r.geo, r.bf, r.grid, r.sp, r.mcc = f[:5]
        r.n = len(arrs[0])
        for k in range(6):
            r.xyzv[k] = _ptr(arrs[k])
        r.q = _ptr(q)
        r.weight = rp.weight if weight is None else weight
        r.seed = rp.seed if seed is None else seed
        r.dt = rp.dt if dt is None else dt
        r.window_steps, r.rel_tol, r.min_events, r.max_steps = window_steps, rel_tol, min_events, max_steps
        r.ne_windows = ne_windows
        return r, (f, arrs, q)

    def calibrate(self, rp, state, flow_target, power_target_W, tol=0.1, max_iter=8, E=None, ne_cells=None,
                  window_steps=256, rel_tol=0.02, min_events=400, max_steps=4096, weight=None, seed=None, dt=None,
                  ne_windows=0):
        """Queue a calibration job (ecris_server_calibrate): runs of rp with
        the weight and rp.Te_warm_eV adjusted until the last window's flow and
        power meet the targets within tol.  Returns the job handle."""
        r, keep = self._request(rp, state, E, ne_cells, window_steps, rel_tol, min_events, max_steps, weight, seed,
                                dt, ne_windows)
        c = CalibRequest()
        c.base = r
        c.flow_target, c.power_target_W, c.tol, c.max_iter = flow_target, power_target_W, tol, max_iter
        j = ctypes.c_int64(0)
        st = ecris_server_calibrate(self.s, ctypes.byref(c), ctypes.byref(j))
        if st != ECRIS_OK:
            raise EcrisError(st, ecris_server_last_error(self.s).decode())
        return j.value

    def calib_poll(self, job):
        res = CalibResult()
        st = ecris_server_calib_poll(self.s, int(job), ctypes.byref(res))
        if st != ECRIS_OK:
            raise EcrisError(st, ecris_server_last_error(self.s).decode())
        k = res.iterations
        return {"state": res.state, "met": bool(res.met), "iterations": k,
                "weight": np.array(res.weight[:k]), "Te_warm_eV": np.array(res.Te_warm_eV[:k]),
                "flow_per_s": np.array(res.flow_per_s[:k]), "power_W": np.array(res.power_W[:k]),
                "steps": np.array(res.steps[:k]), "error": res.error.decode()}

    def submit(self, rp, state, E=None, ne_cells=None, window_steps=256, rel_tol=0.02, min_events=400,
               max_steps=4096, weight=None, seed=None, dt=None, ne_windows=0):
        """Queue a run (ecris_server_submit); ne_windows > 0 makes its n_e
        self-consistent, updated after every ne_windows windows.  Returns the
        ticket."""
        r, keep = self._request(rp, state, E, ne_cells, window_steps, rel_tol, min_events, max_steps, weight, seed,
                                dt, ne_windows)
        t = ctypes.c_int64(0)
        st = ecris_server_submit(self.s, ctypes.byref(r), ctypes.byref(t))
        if st != ECRIS_OK:
            raise EcrisError(st, ecris_server_last_error(self.s).decode())
        return t.value

    def poll(self, ticket):
        res = Result()
        st = ecris_server_poll(self.s, int(ticket), ctypes.byref(res))
        if st != ECRIS_OK:
            raise EcrisError(st, ecris_server_last_error(self.s).decode())
        q1 = res.qmax + 1
        return {"state": res.state, "converged": bool(res.converged), "steps": res.steps,
                "t_submit": res.t_submit, "t_admit": res.t_admit, "t_done": res.t_done,
                "extracted": np.array(res.extracted[:q1]), "lost": np.array(res.lost[:q1]),
                "current_A": np.array(res.current_A[:q1]), "power_W": res.power_W,
                "ke_lost_eV": res.ke_lost_eV, "error": res.error.decode(), "flow_per_s": res.flow_per_s,
                "power_window_W": res.power_window_W}

    def stats(self):
        now = ctypes.c_double()
        qd, rn, dn = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        ist = ctypes.c_double()
        ecris_server_stats(self.s, ctypes.byref(now), ctypes.byref(qd), ctypes.byref(rn), ctypes.byref(dn),
                           ctypes.byref(ist))
        tn = ctypes.c_int64()
        ecris_server_tunings(self.s, ctypes.byref(tn))
        return {"now": now.value, "queued": qd.value, "running": rn.value, "done": dn.value,
                "ion_steps": ist.value, "tunings": tn.value}


FPTD_BINS = 120   # ECRIS_FPTD_BINS


def _fptd(qmax, call):
    hist = np.zeros((qmax + 1, FPTD_BINS), dtype=np.uint64)
    age_sum = np.zeros(qmax + 1, dtype=np.uint64)
    call(_ptr(hist), _ptr(age_sum))
    return {"hist": hist, "age_sum": age_sum}


def _probe_spec(cells, screens, pixels):
    """ecris_probe_spec for the cell list and the (z_lo, z_hi) slabs; the
    cell array is returned with it and must outlive the call."""
    c = np.ascontiguousarray([] if cells is None else cells, dtype=np.uint32)
    sp = ProbeSpec()
    sp.ncells = len(c)
    sp.cells = c.ctypes.data if len(c) else None
    sp.nscreens = len(screens)
    for k, (lo, hi) in enumerate(screens):
        sp.z_lo[k], sp.z_hi[k] = float(lo), float(hi)
    sp.pixels = int(pixels)
    return sp, c


def _probes(qmax, ncells, nscreens, pixels, call):
    qs = qmax + 1
    n = ctypes.c_uint64(0)
    mom = np.zeros((ncells, qs, 7), dtype=np.float64)
    scr = np.zeros((nscreens, qs, pixels, pixels), dtype=np.uint64)
    call(ctypes.byref(n), _ptr(mom) if ncells else None, _ptr(scr) if nscreens else None)
    return {"samples": int(n.value), "moments": mom, "screens": scr}


def _radius(qmax, call):
    r = np.zeros(qmax + 1, dtype=np.float64)
    call(_ptr(r))
    return r


def _cells(nc, call):
    out = {k: np.zeros(nc, dtype=np.float32) for k in ("ne", "delta_x", "delta_y")}
    call(_ptr(out["ne"]), _ptr(out["delta_x"]), _ptr(out["delta_y"]))
    return out


class Run:
    """One ECRIS run on one GPU: fields, particles, steps and diagnostics."""

    def __init__(self, rp, E=None, ne_cells=None, device=0, stream=None):
        self.rp = rp
        self.ctx = ctypes.c_void_p()
        st = ecris_create(ctypes.byref(self.ctx), int(device), stream)
        if st != ECRIS_OK:
            raise EcrisError(st, ecris_last_error(None).decode())
        self._keep = []
        self.init_fields(rp, E, ne_cells)

    def close(self):
        if self.ctx:
            ecris_destroy(self.ctx)
            self.ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_fields(self, rp, E=None, ne_cells=None):
        f = field_structs(rp, E, ne_cells)
        check(self.ctx, ecris_init_fields(self.ctx, *[ctypes.byref(x) for x in f[:5]]))
        self.ncells = rp.nx * rp.ny * rp.nz
        self.qmax = rp.species.qmax

    def load(self, state, weight=None, seed=None):
        """state: dict of x,y,z,vx,vy,vz (float32) and q (uint8), numpy or torch CUDA."""
        rp = self.rp
        arrs = [state[k] for k in ("x", "y", "z", "vx", "vy", "vz")]
        q = state["q"]
        dev = _is_device(arrs[0])
        if not dev:
            arrs = [np.ascontiguousarray(a, dtype=np.float32) for a in arrs]
            q = np.ascontiguousarray(q, dtype=np.uint8)
        self._keep = arrs + [q]
        n = len(arrs[0])
        ptrs = (ctypes.c_void_p * 6)(*[_ptr(a) for a in arrs])
        check(self.ctx, ecris_load_ions(self.ctx, n, ptrs, _ptr(q),
                                        rp.weight if weight is None else weight,
                                        rp.seed if seed is None else seed, 1 if dev else 0))
        self.n = n

    def step(self, nsteps=1, dt=None):
        check(self.ctx, ecris_step(self.ctx, int(nsteps), self.rp.dt if dt is None else dt))

    def diag(self, grids=False):
        return _diag(self.qmax, self.ncells, lambda o: check(self.ctx, ecris_diag(self.ctx, o)), grids)

    def state(self):
        return _state(self.n, lambda p, m: check(self.ctx, ecris_get_state(self.ctx, p, m, 0)))

    def update_ne(self):
        """n_e of every cell := the time-averaged ion charge density since the
        load or the previous call; delta rebuilt from it."""
        check(self.ctx, ecris_update_ne(self.ctx))

    def extraction_radius(self):
        """Summed radius (m) of the extracted ions at the aperture plane, by Q."""
        return _radius(self.qmax, lambda a: check(self.ctx, ecris_get_extraction_radius(self.ctx, a)))

    def set_probes(self, cells=None, screens=(), pixels=256):
        """Install moment probes on the listed cells and x-y screens on the
        (z_lo, z_hi) slabs, pixels x pixels each; zeroes their sums."""
        sp, keep = _probe_spec(cells, screens, pixels)
        check(self.ctx, ecris_set_probes(self.ctx, ctypes.byref(sp)))
        self._probe_shape = (len(keep), len(screens), int(pixels))

    def probe_sample(self):
        """Add the particles as they are now to the probes' sums."""
        check(self.ctx, ecris_probe_sample(self.ctx))

    def probes(self):
        """samples, moments [cell, Q, 7] (count, sum v, sum v^2) and screens [s, Q, py, px]."""
        nc, ns, px = self._probe_shape
        return _probes(self.qmax, nc, ns, px, lambda a, b, c: check(self.ctx, ecris_get_probes(self.ctx, a, b, c)))

    def fptd(self):
        """First-passage times of the extracted ions since the load: hist
        [Q, bin] (bins of ECRIS_FPTD_BINS, 4 per octave of the age in steps)
        and age_sum [Q] (steps)."""
        return _fptd(self.qmax, lambda a, b: check(self.ctx, ecris_get_fptd(self.ctx, a, b)))

    def cells(self):
        """The per-cell electron data the kernels read: n_e (m^-3), delta_x, delta_y."""
        return _cells(self.ncells, lambda a, b, c: check(self.ctx, ecris_get_cells(self.ctx, a, b, c)))

    def set_tuning(self, sort_every=32):
        t = Tuning()
        t.sort_every = int(sort_every)
        check(self.ctx, ecris_set_tuning(self.ctx, ctypes.byref(t)))

    def set_profiling(self, on=True):
        check(self.ctx, ecris_set_profiling(self.ctx, 1 if on else 0))

    def profile(self):
        p = Profile()
        check(self.ctx, ecris_get_profile(self.ctx, ctypes.byref(p)))
        return {f: getattr(p, f) for f, _ in Profile._fields_}

    def state_to_device(self, out):
        """Copy the state into torch CUDA tensors out[x..vz] (float32) and out['meta'] (int32)."""
        ptrs = (ctypes.c_void_p * 6)(*[_ptr(out[k]) for k in ("x", "y", "z", "vx", "vy", "vz")])
        check(self.ctx, ecris_get_state(self.ctx, ptrs, _ptr(out.get("meta")), 1))
