"""ctypes binding of the SIC C ABI (include/sic.h), same names, argument marshalling only.

Importing this module loads ``_build/libsic.so``; it raises ImportError when
the library has not been built: there is no CPU fallback.  Every step of the
path runs in the library's CUDA kernels.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libsic.so")

SIC_OK = 0
SIC_EINVAL = -1
SIC_ENOMEM = -2
SIC_ECUDA = -3
SIC_ERANGE = -4
SIC_ESEGMENT_LONG = -5
SIC_ETIMEOUT = -6
SIC_EBUSY = -7
SIC_ELIMIT = -8
SIC_NX_MAX = 8192

# every symbol include/sic.h declares
EXPORTS = [
    "sic_create", "sic_create_horizontal", "sic_deposit", "sic_field", "sic_push", "sic_step",
    "sic_step_batch", "sic_diagnostics", "sic_history", "sic_get_state", "sic_device_state",
    "sic_sync", "sic_destroy", "sic_strerror", "sic_launch_count",
    "sic_batch_create", "sic_batch_step", "sic_batch_segments", "sic_batch_destroy",
    "sic_server_create", "sic_server_submit", "sic_server_submit_horizontal", "sic_server_tick",
    "sic_server_results", "sic_server_clock", "sic_server_stats", "sic_server_destroy",
    "sic_step_batch_static", "sic_moments", "sic_refine", "sic_sheet_counts", "sic_batch_autotune",
    "sic_run", "sic_mode_history", "sic_spectrum",
]


class sic_config(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32),
        ("box_length", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("n_sheets", ctypes.c_int32),
        ("tracers_per_sheet", ctypes.POINTER(ctypes.c_int32)),
        ("sheet_closed", ctypes.POINTER(ctypes.c_uint8)),
        ("sheet_winding", ctypes.POINTER(ctypes.c_int32)),
        ("charge_to_mass", ctypes.c_double),
        ("half_step_init", ctypes.c_int32),
        ("strict_segments", ctypes.c_int32),
        ("history_len", ctypes.c_int32),
        ("stream", ctypes.c_void_p),
        ("deposit", ctypes.c_int32),
        ("refine_length", ctypes.c_double),
        ("refine_split", ctypes.c_double),
        ("max_tracers", ctypes.c_int64),
        ("charge_unit", ctypes.c_double),
        ("mode_k", ctypes.c_int32),
    ]


class sic_diag(ctypes.Structure):
    _fields_ = [
        ("step", ctypes.c_int64),
        ("t", ctypes.c_double),
        ("field_energy", ctypes.c_double),
        ("kinetic_energy", ctypes.c_double),
        ("momentum", ctypes.c_double),
        ("charge_fixed", ctypes.c_int64),
        ("charge_unit", ctypes.c_double),
        ("max_segment", ctypes.c_double),
    ]


class sic_server_config(ctypes.Structure):
    _fields_ = [
        ("hbm_budget", ctypes.c_int64),
        ("max_active", ctypes.c_int32),
        ("chunk_steps", ctypes.c_int32),
        ("plain", ctypes.c_int32),
        ("stream", ctypes.c_void_p),
    ]


class sic_result(ctypes.Structure):
    _fields_ = [
        ("id", ctypes.c_int64),
        ("status", ctypes.c_int32),
        ("pad", ctypes.c_int32),
        ("steps", ctypes.c_int64),
        ("segment_updates", ctypes.c_int64),
        ("field_energy", ctypes.c_double),
        ("kinetic_energy", ctypes.c_double),
        ("momentum", ctypes.c_double),
        ("charge_fixed", ctypes.c_int64),
        ("t_submit", ctypes.c_double),
        ("t_admit", ctypes.c_double),
        ("t_done", ctypes.c_double),
        ("sim", ctypes.c_void_p),
    ]


class sic_server_info(ctypes.Structure):
    _fields_ = [
        ("bytes_in_use", ctypes.c_int64),
        ("bytes_peak", ctypes.c_int64),
        ("hbm_budget", ctypes.c_int64),
        ("active", ctypes.c_int32),
        ("queued", ctypes.c_int32),
        ("completed", ctypes.c_int64),
        ("segment_updates", ctypes.c_int64),
        ("ticks", ctypes.c_int64),
        ("busy_s", ctypes.c_double),
        ("waits_slots", ctypes.c_int64),
        ("waits_memory", ctypes.c_int64),
        ("refinements", ctypes.c_int64),
    ]


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"SIC CUDA library not built: {path} (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER
    dp, ip, lp, vp = P(ctypes.c_double), P(ctypes.c_int32), P(ctypes.c_int64), ctypes.c_void_p
    simp = vp
    sig = {
        "sic_create": ([P(sic_config), dp, dp, dp, P(simp)], ctypes.c_int),
        "sic_create_horizontal": ([P(sic_config), ctypes.c_int32, dp, dp, dp, P(simp)], ctypes.c_int),
        "sic_deposit": ([simp, lp, dp], ctypes.c_int),
        "sic_field": ([simp, dp], ctypes.c_int),
        "sic_push": ([simp], ctypes.c_int),
        "sic_step": ([simp, ctypes.c_int32], ctypes.c_int),
        "sic_run": ([simp, ctypes.c_int32, lp], ctypes.c_int),
        "sic_step_batch": ([P(simp), ctypes.c_int32, ip], ctypes.c_int),
        "sic_step_batch_static": ([P(simp), ctypes.c_int32, ip], ctypes.c_int),
        "sic_moments": ([simp, ctypes.c_int32, dp, dp], ctypes.c_int),
        "sic_batch_autotune": ([vp, ctypes.c_int32, ip, ip, ip], ctypes.c_int),
        "sic_refine": ([simp, ctypes.c_double, lp], ctypes.c_int),
        "sic_sheet_counts": ([simp, ip], ctypes.c_int),
        "sic_diagnostics": ([simp, P(sic_diag)], ctypes.c_int),
        "sic_history": ([simp, dp, ctypes.c_int32, ip], ctypes.c_int),
        "sic_mode_history": ([simp, dp, ctypes.c_int32, ip], ctypes.c_int),
        "sic_spectrum": ([simp, ctypes.c_int32, dp], ctypes.c_int),
        "sic_get_state": ([simp, dp, dp], ctypes.c_int),
        "sic_device_state": ([simp, P(vp), P(vp), P(vp)], ctypes.c_int),
        "sic_sync": ([simp], ctypes.c_int),
        "sic_destroy": ([simp], None),
        "sic_strerror": ([ctypes.c_int], ctypes.c_char_p),
        "sic_launch_count": ([], ctypes.c_int64),
        "sic_batch_create": ([P(simp), ctypes.c_int32, P(vp)], ctypes.c_int),
        "sic_batch_step": ([vp, ctypes.c_int32], ctypes.c_int),
        "sic_batch_segments": ([vp], ctypes.c_int64),
        "sic_batch_destroy": ([vp], None),
        "sic_server_create": ([P(sic_server_config), P(vp)], ctypes.c_int),
        "sic_server_submit": ([vp, P(sic_config), dp, dp, dp, ctypes.c_int32, ctypes.c_int32,
                               P(ctypes.c_int64)], ctypes.c_int),
        "sic_server_submit_horizontal": ([vp, P(sic_config), ctypes.c_int32, dp, dp, dp, ctypes.c_int32,
                                          ctypes.c_int32, P(ctypes.c_int64)], ctypes.c_int),
        "sic_server_tick": ([vp, ip], ctypes.c_int),
        "sic_server_results": ([vp, P(sic_result), ctypes.c_int32, ip], ctypes.c_int),
        "sic_server_clock": ([vp], ctypes.c_double),
        "sic_server_stats": ([vp, P(sic_server_info)], ctypes.c_int),
        "sic_server_destroy": ([vp], None),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


_lib = load_library()


class SicError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {_lib.sic_strerror(code).decode()} ({code})")


def _check(code: int, what: str):
    if code != SIC_OK:
        raise SicError(code, what)


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def sic_strerror(code: int) -> str:
    return _lib.sic_strerror(code).decode()


def sic_launch_count() -> int:
    return int(_lib.sic_launch_count())


def _config(nx, L, dt, n_sheets, counts=None, closed=None, winding=None, qm=1.0,
            half_step_init=True, strict=False, history_len=1, stream=None, order=0, refine=0.0,
            refine_split=0.0, max_tracers=0, charge_unit=0.0, mode_k=0):
    cfg = sic_config()
    cfg.nx = int(nx)
    cfg.box_length = float(L)
    cfg.dt = float(dt)
    cfg.n_sheets = int(n_sheets)
    keep = []
    if counts is not None:
        c = np.ascontiguousarray(counts, dtype=np.int32)
        cl = np.ascontiguousarray(closed, dtype=np.uint8)
        wd = np.ascontiguousarray(winding if winding is not None else np.zeros(n_sheets), dtype=np.int32)
        keep += [c, cl, wd]
        cfg.tracers_per_sheet = c.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        cfg.sheet_closed = cl.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
        cfg.sheet_winding = wd.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    cfg.charge_to_mass = float(qm)
    cfg.half_step_init = int(bool(half_step_init))
    cfg.strict_segments = int(bool(strict))
    cfg.history_len = int(history_len)
    cfg.stream = ctypes.c_void_p(int(stream) if stream else 0)
    cfg.deposit = int(order)
    cfg.refine_length = float(refine)
    cfg.refine_split = float(refine_split) if refine else 0.0
    cfg.max_tracers = int(max_tracers)
    cfg.charge_unit = float(charge_unit)
    cfg.mode_k = int(mode_k)
    return cfg, keep


class Sim:
    """One simulation held on the GPU (wraps a ``sic_sim*``)."""

    def __init__(self, handle, nx, n_tracers, counts):
        self._h = handle
        self.nx = int(nx)
        self.n_tracers = int(n_tracers)
        self.counts = np.asarray(counts, dtype=np.int64)

    # -- construction -------------------------------------------------------
    @classmethod
    def sic_create(cls, nx, L, dt, counts, closed, winding, x, v, w, qm=1.0, half_step_init=True,
                   strict=False, history_len=1, stream=None, order=0, refine=0.0, refine_split=0.0,
                   max_tracers=0, charge_unit=0.0, mode_k=0):
        counts = np.ascontiguousarray(counts, dtype=np.int32)
        cfg, keep = _config(nx, L, dt, counts.size, counts, closed, winding, qm, half_step_init,
                            strict, history_len, stream, order, refine, refine_split, max_tracers, charge_unit,
                            mode_k)
        x = np.ascontiguousarray(x, dtype=np.float64)
        v = np.ascontiguousarray(v, dtype=np.float64)
        w = np.ascontiguousarray(w, dtype=np.float64)
        n = int(counts.sum())
        if x.size != n or v.size != n or w.size != n:
            raise ValueError("x, v and w need one entry per tracer")
        h = ctypes.c_void_p()
        _check(_lib.sic_create(ctypes.byref(cfg), _dptr(x), _dptr(v), _dptr(w), ctypes.byref(h)),
               "sic_create")
        return cls(h, nx, n, counts)

    @classmethod
    def sic_create_horizontal(cls, nx, L, dt, x_template, v_sheet, w_sheet, qm=1.0,
                              half_step_init=True, strict=False, history_len=1, stream=None, order=0,
                              refine=0.0, refine_split=0.0, max_tracers=0, mode_k=0):
        xt = np.ascontiguousarray(x_template, dtype=np.float64)
        vs = np.ascontiguousarray(v_sheet, dtype=np.float64)
        ws = np.ascontiguousarray(w_sheet, dtype=np.float64)
        if vs.shape != ws.shape:
            raise ValueError("v_sheet and w_sheet need one entry per sheet")
        cfg, keep = _config(nx, L, dt, vs.size, None, None, None, qm, half_step_init, strict,
                            history_len, stream, order, refine, refine_split, max_tracers, 0.0, mode_k)
        h = ctypes.c_void_p()
        _check(_lib.sic_create_horizontal(ctypes.byref(cfg), xt.size, _dptr(xt), _dptr(vs), _dptr(ws),
                                          ctypes.byref(h)), "sic_create_horizontal")
        return cls(h, nx, xt.size * vs.size, np.full(vs.size, xt.size))

    @classmethod
    def from_problem(cls, p, history_len=None, strict=False, stream=None, horizontal=None, order=0,
                     refine=None, mode_k=0):
        """Create from an ``inputs.Problem`` (compact form when it has one); order
        is the deposit (SIC_DEPOSIT_*): 0 box particles, 1 piecewise linear
        (Sec. 2.5), 2 and 3 PIC nearest grid point and cloud in cell; refine is
        the refinement length (default: the problem's own); mode_k the Fourier
        mode whose field energy every step records (0: none)."""
        hl = history_len if history_len is not None else max(1, p.n_steps)
        if refine is None:
            refine = p.refine_length if order in (0, 1, 4) else 0.0
        split = p.refine_split if refine == p.refine_length else 0.0
        if horizontal is None:
            horizontal = p.is_horizontal
        if horizontal:
            return cls.sic_create_horizontal(p.nx, p.L, p.dt, p.x_template, p.v_sheet, p.w_sheet,
                                             qm=p.qm, half_step_init=p.half_step_init, strict=strict,
                                             history_len=hl, stream=stream, order=order, refine=refine,
                                             refine_split=split, max_tracers=p.max_tracers, mode_k=mode_k)
        return cls.sic_create(p.nx, p.L, p.dt, p.counts, p.closed, p.winding, p.x, p.v, p.w,
                              qm=p.qm, half_step_init=p.half_step_init, strict=strict,
                              history_len=hl, stream=stream, order=order, refine=refine, refine_split=split,
                              max_tracers=p.max_tracers, mode_k=mode_k)

    # -- the C ABI, one method per entry point ------------------------------
    @property
    def handle(self):
        if self._h is None:
            raise ValueError("simulation destroyed")
        return self._h

    def sic_deposit(self):
        mesh = np.zeros(self.nx, dtype=np.int64)
        rho = np.zeros(self.nx, dtype=np.float64)
        _check(_lib.sic_deposit(self.handle, mesh.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                _dptr(rho)), "sic_deposit")
        return mesh, rho

    def sic_moments(self, weighting=0):
        """(n, j): number and current density, zero order on cells (0) or first
        order on nodes (1)."""
        n = np.zeros(self.nx, dtype=np.float64)
        j = np.zeros(self.nx, dtype=np.float64)
        _check(_lib.sic_moments(self.handle, int(weighting), _dptr(n), _dptr(j)), "sic_moments")
        return n, j

    def sic_refine(self, l_ref):
        """Split every particle longer than l_ref at its centre (Sec. 2.6);
        returns the number of new tracers and updates ``counts``."""
        added = ctypes.c_int64()
        _check(_lib.sic_refine(self.handle, float(l_ref), ctypes.byref(added)), "sic_refine")
        counts = np.zeros(self.counts.size, dtype=np.int32)
        _check(_lib.sic_sheet_counts(self.handle, counts.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))),
               "sic_sheet_counts")
        self.counts = counts.astype(np.int64)
        self.n_tracers = int(counts.sum())
        return int(added.value)

    def sic_field(self):
        E = np.zeros(self.nx, dtype=np.float64)
        _check(_lib.sic_field(self.handle, _dptr(E)), "sic_field")
        return E

    def sic_push(self):
        _check(_lib.sic_push(self.handle), "sic_push")

    def sic_step(self, n_steps: int):
        _check(_lib.sic_step(self.handle, int(n_steps)), "sic_step")

    def sic_run(self, n_steps: int):
        """n_steps steps, refining whenever a particle outgrows the refinement
        length (Sec. 2.6); returns the number of tracers added."""
        added = ctypes.c_int64()
        _check(_lib.sic_run(self.handle, int(n_steps), ctypes.byref(added)), "sic_run")
        self._update_counts()
        return int(added.value)

    def _update_counts(self):
        counts = np.zeros(self.counts.size, dtype=np.int32)
        _check(_lib.sic_sheet_counts(self.handle, counts.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))),
               "sic_sheet_counts")
        self.counts = counts.astype(np.int64)
        self.n_tracers = int(counts.sum())

    def sic_diagnostics(self) -> dict:
        d = sic_diag()
        _check(_lib.sic_diagnostics(self.handle, ctypes.byref(d)), "sic_diagnostics")
        return {name: getattr(d, name) for name, _ in sic_diag._fields_}

    def sic_history(self, history_len: int):
        """The last min(history_len, ring length, steps) rows [W_E, KE, P, Q]."""
        buf = np.zeros((max(1, int(history_len)), 4), dtype=np.float64)
        rows = ctypes.c_int32()
        _check(_lib.sic_history(self.handle, _dptr(buf), buf.shape[0], ctypes.byref(rows)), "sic_history")
        return buf[: rows.value]

    def sic_mode_history(self, history_len: int):
        """The last min(history_len, ring length, steps) values of the field
        energy in Fourier mode mode_k (Sec. 3.2), one per history row."""
        buf = np.zeros(max(1, int(history_len)), dtype=np.float64)
        rows = ctypes.c_int32()
        _check(_lib.sic_mode_history(self.handle, _dptr(buf), buf.size, ctypes.byref(rows)), "sic_mode_history")
        return buf[: rows.value]

    def sic_spectrum(self, field=0):
        """|X^_k|, k = 0 .. nx/2, of the latest deposit's density (field 0) or
        node field (field 1)."""
        out = np.zeros(self.nx // 2 + 1, dtype=np.float64)
        _check(_lib.sic_spectrum(self.handle, int(field), _dptr(out)), "sic_spectrum")
        return out

    def sic_get_state(self):
        x = np.zeros(self.n_tracers, dtype=np.float64)
        v = np.zeros(self.n_tracers, dtype=np.float64)
        _check(_lib.sic_get_state(self.handle, _dptr(x), _dptr(v)), "sic_get_state")
        return x, v

    def sic_device_state(self):
        """(positions uint32* in the SIC position format, velocities float*,
        sheet offsets) as integer addresses."""
        pu, pv, po = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        _check(_lib.sic_device_state(self.handle, ctypes.byref(pu), ctypes.byref(pv),
                                     ctypes.byref(po)), "sic_device_state")
        offs = np.ctypeslib.as_array(ctypes.cast(po, ctypes.POINTER(ctypes.c_int64)),
                                     shape=(self.counts.size,)).copy()
        return pu.value, pv.value, offs

    def sic_sync(self):
        _check(_lib.sic_sync(self.handle), "sic_sync")

    def sic_destroy(self):
        if self._h is not None:
            _lib.sic_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.sic_destroy()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.sic_destroy()


def sic_step_batch(sims, n_steps):
    arr = (ctypes.c_void_p * len(sims))(*[s.handle for s in sims])
    steps = np.ascontiguousarray(n_steps, dtype=np.int32)
    if steps.size != len(sims):
        raise ValueError("one step count per simulation")
    _check(_lib.sic_step_batch(arr, len(sims), steps.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))),
           "sic_step_batch")


SIC_STATIC_MAX_SIMS = 64
SIC_AUTOTUNE_CANDIDATES = 10
SIC_DEPOSIT_BOX, SIC_DEPOSIT_LINEAR, SIC_DEPOSIT_PIC_NGP, SIC_DEPOSIT_PIC_CIC, SIC_DEPOSIT_FIRST = 0, 1, 2, 3, 4


def sic_step_batch_static(sims, n_steps):
    """``sic_step_batch`` with the launch plan in the library's fixed device
    scratch: no allocation; at most SIC_STATIC_MAX_SIMS simulations."""
    arr = (ctypes.c_void_p * len(sims))(*[s.handle for s in sims])
    steps = np.ascontiguousarray(n_steps, dtype=np.int32)
    if steps.size != len(sims):
        raise ValueError("one step count per simulation")
    _check(_lib.sic_step_batch_static(arr, len(sims), steps.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))),
           "sic_step_batch_static")


class Batch:
    """A persistent batch of simulations stepped together (``sic_batch*``)."""

    def __init__(self, sims):
        arr = (ctypes.c_void_p * len(sims))(*[s.handle for s in sims])
        h = ctypes.c_void_p()
        _check(_lib.sic_batch_create(arr, len(sims), ctypes.byref(h)), "sic_batch_create")
        self._h = h
        self.sims = list(sims)

    def sic_batch_step(self, n_steps):
        _check(_lib.sic_batch_step(self._h, int(n_steps)), "sic_batch_step")

    def sic_batch_autotune(self, steps_each=3):
        """Time the schedule candidates on real steps and keep the fastest;
        advances every member by SIC_AUTOTUNE_CANDIDATES (steps_each + 1)
        steps.  Returns (claim divisor, staging, smallest claim)."""
        d, st, mn = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(_lib.sic_batch_autotune(self._h, int(steps_each), ctypes.byref(d), ctypes.byref(st),
                                       ctypes.byref(mn)), "sic_batch_autotune")
        return d.value, st.value, mn.value

    def sic_batch_segments(self):
        return int(_lib.sic_batch_segments(self._h))

    def sic_batch_destroy(self):
        if self._h is not None:
            _lib.sic_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.sic_batch_destroy()
        except Exception:
            pass


class Server:
    """The request server (``sic_server*``): continuous batching of simulations."""

    def __init__(self, hbm_budget=64 << 30, max_active=64, chunk_steps=32, plain=False, stream=None):
        cfg = sic_server_config()
        cfg.hbm_budget = int(hbm_budget)
        cfg.max_active = int(max_active)
        cfg.chunk_steps = int(chunk_steps)
        cfg.plain = int(bool(plain))
        cfg.stream = ctypes.c_void_p(int(stream) if stream else 0)
        h = ctypes.c_void_p()
        _check(_lib.sic_server_create(ctypes.byref(cfg), ctypes.byref(h)), "sic_server_create")
        self._h = h

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("server destroyed")
        return self._h

    def sic_server_submit_horizontal(self, p, n_steps=None, keep=False, history_len=1):
        """Queue an ``inputs.Problem`` with horizontal sheets; returns the request id."""
        xt = np.ascontiguousarray(p.x_template, dtype=np.float64)
        vs = np.ascontiguousarray(p.v_sheet, dtype=np.float64)
        ws = np.ascontiguousarray(p.w_sheet, dtype=np.float64)
        cfg, keepalive = _config(p.nx, p.L, p.dt, vs.size, None, None, None, p.qm, p.half_step_init,
                                 history_len=history_len, refine=p.refine_length, refine_split=p.refine_split,
                                 max_tracers=p.max_tracers)
        rid = ctypes.c_int64()
        _check(_lib.sic_server_submit_horizontal(self.handle, ctypes.byref(cfg), xt.size, _dptr(xt), _dptr(vs),
                                                 _dptr(ws), int(p.n_steps if n_steps is None else n_steps),
                                                 int(bool(keep)), ctypes.byref(rid)),
               "sic_server_submit_horizontal")
        return rid.value

    def sic_server_submit(self, p, n_steps=None, keep=False):
        """Queue an ``inputs.Problem`` from its full per-tracer arrays."""
        x = np.ascontiguousarray(p.x, dtype=np.float64)
        v = np.ascontiguousarray(p.v, dtype=np.float64)
        w = np.ascontiguousarray(p.w, dtype=np.float64)
        cfg, keepalive = _config(p.nx, p.L, p.dt, p.counts.size, p.counts, p.closed, p.winding, p.qm,
                                 p.half_step_init, refine=p.refine_length, refine_split=p.refine_split,
                                 max_tracers=p.max_tracers)
        rid = ctypes.c_int64()
        _check(_lib.sic_server_submit(self.handle, ctypes.byref(cfg), _dptr(x), _dptr(v), _dptr(w),
                                      int(p.n_steps if n_steps is None else n_steps), int(bool(keep)),
                                      ctypes.byref(rid)), "sic_server_submit")
        return rid.value

    def sic_server_tick(self):
        pending = ctypes.c_int32()
        _check(_lib.sic_server_tick(self.handle, ctypes.byref(pending)), "sic_server_tick")
        return pending.value

    def sic_server_results(self, max_results=4096):
        buf = (sic_result * max_results)()
        n = ctypes.c_int32()
        _check(_lib.sic_server_results(self.handle, buf, max_results, ctypes.byref(n)), "sic_server_results")
        out = []
        for i in range(n.value):
            r = {name: getattr(buf[i], name) for name, _ in sic_result._fields_ if name not in ("pad", "sim")}
            r["sim"] = buf[i].sim
            out.append(r)
        return out

    def sic_server_clock(self):
        return float(_lib.sic_server_clock(self.handle))

    def sic_server_stats(self):
        info = sic_server_info()
        _check(_lib.sic_server_stats(self.handle, ctypes.byref(info)), "sic_server_stats")
        return {name: getattr(info, name) for name, _ in sic_server_info._fields_}

    def sic_server_destroy(self):
        if self._h is not None:
            _lib.sic_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.sic_server_destroy()
        except Exception:
            pass


def adopt_sim(handle, nx, counts):
    """Wrap a ``sic_sim*`` a server handed back (result of a keep request)."""
    counts = np.asarray(counts, dtype=np.int64)
    return Sim(ctypes.c_void_p(handle), nx, int(counts.sum()), counts)
