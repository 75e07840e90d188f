"""FP64 CPU oracle of the SIC Vlasov-Poisson step (arXiv:1506.07207).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg use this package; the product path never imports,
links or runs it, and it shares no code with the CUDA path.

The arithmetic lives in ``sic_oracle.c`` (plain double-precision loops, one
function per definition of the paper); this module compiles it with gcc on
first use and wraps it with ctypes.  ``theory`` holds the closed-form
dispersion relations used as pins, ``fits`` the rate fitter.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sic_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libsic_oracle.so")
_lock = threading.Lock()
_lib = None

# -ffp-contract=off: no fused multiply-add contraction, so x86 and Arm hosts
# give the same bits.
CFLAGS = ["-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c99"]


def build(force: bool = False) -> str:
    """Compile ``sic_oracle.c`` into ``_build/libsic_oracle.so``; return its path."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int32)
            bp = ctypes.POINTER(ctypes.c_uint8)
            lib.orc_deposit.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                        ip, bp, ip, dp, dp, dp]
            lib.orc_deposit.restype = ctypes.c_int
            lib.orc_deposit_linear.argtypes = lib.orc_deposit.argtypes
            lib.orc_deposit_seg.argtypes = lib.orc_deposit.argtypes
            lib.orc_deposit_seg.restype = ctypes.c_int
            lib.orc_deposit_linear_seg.argtypes = lib.orc_deposit.argtypes
            lib.orc_deposit_linear_seg.restype = ctypes.c_int
            lib.orc_deposit_linear.restype = ctypes.c_int
            lib.orc_moments.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int, ip, bp, ip,
                                        dp, dp, dp, ctypes.c_int, dp, dp]
            lib.orc_moments.restype = ctypes.c_int
            lib.orc_deposit_pic.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_long, dp, dp,
                                            ctypes.c_int, dp]
            lib.orc_deposit_pic.restype = ctypes.c_int
            lib.orc_field.argtypes = [ctypes.c_int, ctypes.c_double, dp, dp, dp]
            lib.orc_field.restype = None
            lib.orc_field_nodes.argtypes = [ctypes.c_int, ctypes.c_double, dp, dp, dp]
            lib.orc_field_nodes.restype = None
            lib.orc_deposit_first.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                              ip, bp, ip, dp, dp, dp]
            lib.orc_deposit_first.restype = ctypes.c_int
            lib.orc_gather.argtypes = [ctypes.c_int, ctypes.c_double, dp, ctypes.c_long,
                                       dp, dp]
            lib.orc_gather.restype = None
            lib.orc_field_energy.argtypes = [ctypes.c_int, ctypes.c_double, dp]
            lib.orc_field_energy.restype = ctypes.c_double
            lib.orc_run.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                    ip, bp, ip, ctypes.c_long, dp, dp, dp,
                                    ctypes.c_int, dp, dp, dp, ctypes.c_int]
            lib.orc_run.restype = ctypes.c_int
            lp = ctypes.POINTER(ctypes.c_long)
            ip_mut = ctypes.POINTER(ctypes.c_int32)
            lib.orc_refine.argtypes = [ctypes.c_double, ctypes.c_int, ip_mut, bp, ip, ctypes.c_long,
                                       dp, dp, dp, ctypes.c_double]
            lib.orc_refine.restype = ctypes.c_long
            lib.orc_run_refined.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                            ctypes.c_int, ip_mut, bp, ip, ctypes.c_long, dp, dp, dp,
                                            ctypes.c_int, ctypes.c_double, ctypes.c_double, dp, lp]
            lib.orc_run_refined.restype = ctypes.c_int
            _lib = lib
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a, ctype):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _sheets(counts, closed, winding):
    counts = np.ascontiguousarray(counts, dtype=np.int32)
    closed = np.ascontiguousarray(closed, dtype=np.uint8)
    winding = np.ascontiguousarray(winding, dtype=np.int32)
    if not (counts.shape == closed.shape == winding.shape):
        raise ValueError("counts, closed and winding need one entry per sheet")
    return counts, closed, winding


def deposit(nx, L, counts, closed, winding, x, w, order=0):
    """Charge per cell (Eq. overlap and Eq. rho_sum, times dx); order 1 uses
    the piecewise-linear particles of Sec. 2.5, 2 and 3 the PIC point charges
    of the tracers (nearest grid point, cloud in cell), 4 the first-order
    weighting of the particles onto the nodes (Sec. 2.4; charge per node)."""
    lib = _load()
    counts, closed, winding = _sheets(counts, closed, winding)
    x, w = _f64(x), _f64(w)
    if x.shape != w.shape or x.size != int(counts.sum()):
        raise ValueError("x and w need one entry per tracer")
    out = np.zeros(int(nx), dtype=np.float64)
    if order in (2, 3):
        lib.orc_deposit_pic(int(nx), float(L), x.size, _ptr(x, ctypes.c_double), _ptr(w, ctypes.c_double),
                            int(order), _ptr(out, ctypes.c_double))
        return out
    fn = {1: lib.orc_deposit_linear, 4: lib.orc_deposit_first}.get(order, lib.orc_deposit)
    rc = fn(int(nx), float(L), counts.size, _ptr(counts, ctypes.c_int32),
                         _ptr(closed, ctypes.c_uint8), _ptr(winding, ctypes.c_int32),
                         _ptr(x, ctypes.c_double), _ptr(w, ctypes.c_double),
                         _ptr(out, ctypes.c_double))
    if rc:
        raise ValueError("every sheet needs at least two tracers")
    return out


def density(nx, L, counts, closed, winding, x, w, order=0):
    """Cell-averaged number density n_j = charge_j / dx."""
    return deposit(nx, L, counts, closed, winding, x, w, order) / (float(L) / int(nx))


def moments(nx, L, counts, closed, winding, x, v, w, weighting=0):
    """(n, j): number and current density by zero-order (cells, Eq. rho_sum and
    Eq. j_sum) or first-order (nodes, Sec. 2.4) weighting of the particles."""
    lib = _load()
    counts, closed, winding = _sheets(counts, closed, winding)
    x, v, w = _f64(x), _f64(v), _f64(w)
    if not (x.shape == v.shape == w.shape) or x.size != int(counts.sum()):
        raise ValueError("x, v and w need one entry per tracer")
    n = np.zeros(int(nx))
    j = np.zeros(int(nx))
    rc = lib.orc_moments(int(nx), float(L), counts.size, _ptr(counts, ctypes.c_int32),
                         _ptr(closed, ctypes.c_uint8), _ptr(winding, ctypes.c_int32),
                         _ptr(x, ctypes.c_double), _ptr(v, ctypes.c_double), _ptr(w, ctypes.c_double),
                         int(weighting), _ptr(n, ctypes.c_double), _ptr(j, ctypes.c_double))
    if rc:
        raise ValueError("every sheet needs at least two tracers")
    return n, j


def field(nx, L, charge, nodes=False):
    """(rho, E) from the per-cell charge: neutralised density and node field;
    nodes=True takes the charge on the nodes (first-order weighting) and
    integrates between nodes by the trapezoid rule (orc_field_nodes)."""
    lib = _load()
    charge = _f64(charge)
    rho = np.zeros(int(nx))
    E = np.zeros(int(nx))
    fn = lib.orc_field_nodes if nodes else lib.orc_field
    fn(int(nx), float(L), _ptr(charge, ctypes.c_double), _ptr(rho, ctypes.c_double), _ptr(E, ctypes.c_double))
    return rho, E


def gather(nx, L, E, x):
    """Linear-weighting gather of the node field E at positions x."""
    lib = _load()
    E, x = _f64(E), _f64(x)
    out = np.zeros_like(x)
    lib.orc_gather(int(nx), float(L), _ptr(E, ctypes.c_double), x.size,
                   _ptr(x, ctypes.c_double), _ptr(out, ctypes.c_double))
    return out


def field_energy(nx, L, E):
    """W_E = 1/2 sum_j E_j^2 dx."""
    return _load().orc_field_energy(int(nx), float(L), _ptr(_f64(E), ctypes.c_double))


def dft(X, k):
    """X^_k = sum_j X_j exp(-2 pi i j k / nx) of the mesh values X_j, by the
    definition (the phase reduced exactly: j k mod nx)."""
    X = _f64(X)
    nx = X.size
    j = np.arange(nx, dtype=np.int64)
    ph = 2.0 * np.pi * ((j * int(k)) % nx) / nx
    return complex(np.sum(X * np.cos(ph)), -np.sum(X * np.sin(ph)))


def spectrum(X):
    """|X^_k| for k = 0 .. nx/2 (Sec. 3.2 shows the transform of the charge
    density during the linear growth of the two-stream instability)."""
    X = _f64(X)
    return np.array([abs(dft(X, k)) for k in range(X.size // 2 + 1)])


def mode_energy(E, L, k):
    """Field energy in the Fourier mode pair +-k of the node field E (Sec. 3.2,
    the energy in the excited mode): W_k = dx / nx |E^_k|^2 for 0 < k < nx/2
    and half that for k = nx/2, so that for a zero-mean field the W_k of
    k = 1 .. nx/2 add up to W_E = 1/2 sum_j E_j^2 dx (Parseval)."""
    E = _f64(E)
    nx = E.size
    dx = float(L) / nx
    a2 = abs(dft(E, k)) ** 2
    return (0.5 if 2 * int(k) == nx else 1.0) * dx / nx * a2


def run(nx, L, dt, counts, closed, winding, x, v, w, n_steps, qm=1.0,
        half_step_init=True, record_E=False, order=0):
    """Leapfrog SIC run; returns dict(x, v, E, hist[, E_hist]).

    hist has n_steps+1 rows [W_E, KE, P, Q_total]; KE and P are time-centred
    on each step (NaN on the last row).
    """
    lib = _load()
    counts, closed, winding = _sheets(counts, closed, winding)
    x = np.array(x, dtype=np.float64, copy=True)
    v = np.array(v, dtype=np.float64, copy=True)
    w = _f64(w)
    n = x.size
    hist = np.zeros((n_steps + 1, 4))
    e_hist = np.zeros((n_steps + 1, int(nx))) if record_E else None
    E = np.zeros(int(nx))
    rc = lib.orc_run(int(nx), float(L), float(dt), float(qm), int(bool(half_step_init)),
                     counts.size, _ptr(counts, ctypes.c_int32), _ptr(closed, ctypes.c_uint8),
                     _ptr(winding, ctypes.c_int32), n, _ptr(x, ctypes.c_double),
                     _ptr(v, ctypes.c_double), _ptr(w, ctypes.c_double), int(n_steps),
                     _ptr(hist, ctypes.c_double), _ptr(e_hist, ctypes.c_double),
                     _ptr(E, ctypes.c_double), int(order))
    if rc:
        raise ValueError("every sheet needs at least two tracers")
    out = dict(x=x, v=v, E=E, hist=hist)
    if record_E:
        out["E_hist"] = e_hist
    return out


def deposit_seg(nx, L, counts, closed, winding, x, qseg, order=0):
    """Charge per cell of particles whose charges are given per particle:
    qseg[i] belongs to the particle starting at tracer i; order 1 makes them
    piecewise linear (Sec. 2.5)."""
    lib = _load()
    counts, closed, winding = _sheets(counts, closed, winding)
    x, qseg = _f64(x), _f64(qseg)
    out = np.zeros(int(nx))
    fn = lib.orc_deposit_linear_seg if order == 1 else lib.orc_deposit_seg
    rc = fn(int(nx), float(L), counts.size, _ptr(counts, ctypes.c_int32),
                             _ptr(closed, ctypes.c_uint8), _ptr(winding, ctypes.c_int32),
                             _ptr(x, ctypes.c_double), _ptr(qseg, ctypes.c_double), _ptr(out, ctypes.c_double))
    if rc:
        raise ValueError("every sheet needs at least two tracers")
    return out


def particle_charges(counts, closed, w):
    """Per-particle charges q_s = (w_i + w_{i+1}) / 2 of tracer weights, in the
    layout of deposit_seg (0 after the last tracer of an open sheet)."""
    w = _f64(w)
    q = np.zeros_like(w)
    base = 0
    for n, c in zip(counts, closed):
        ws = w[base:base + n]
        q[base:base + n - 1] = 0.5 * (ws[:-1] + ws[1:])
        q[base + n - 1] = 0.5 * (ws[-1] + ws[0]) if c else 0.0
        base += n
    return q


def refine(L, counts, closed, winding, x, v, qseg, l_ref):
    """One pass of the refinement of Sec. 2.6: every particle longer than
    l_ref gets a new tracer at its centre, with the mean velocity of its two
    tracers; each half carries half the charge.  Returns the new
    (counts, x, v, qseg)."""
    xs, vs, qs, cs = [], [], [], []
    base = 0
    for n, c, wd in zip(counts, closed, winding):
        xo, vo, qo = x[base:base + n], v[base:base + n], qseg[base:base + n]
        nx_, nv_, nq_ = [], [], []
        for i in range(n):
            last = i + 1 == n
            if last and not c:
                nx_.append(xo[i]); nv_.append(vo[i]); nq_.append(qo[i])
                break
            xb = xo[0] + wd * L if last else xo[i + 1]
            vb = vo[0] if last else vo[i + 1]
            if abs(xb - xo[i]) > l_ref:
                nx_ += [xo[i], 0.5 * (xo[i] + xb)]
                nv_ += [vo[i], 0.5 * (vo[i] + vb)]
                nq_ += [0.5 * qo[i], 0.5 * qo[i]]
            else:
                nx_.append(xo[i]); nv_.append(vo[i]); nq_.append(qo[i])
        xs.append(nx_); vs.append(nv_); qs.append(nq_); cs.append(len(nx_))
        base += n
    cat = lambda a: np.array([t for part in a for t in part], dtype=np.float64)
    return np.array(cs, dtype=np.int32), cat(xs), cat(vs), cat(qs)


def run_refined(nx, L, dt, counts, closed, winding, x, v, qseg, n_steps, l_ref, every, qm=1.0):
    """Leapfrog run of box particles with per-particle charges, refined
    (``refine``) after every ``every`` steps.  The velocities are v^{-1/2} on
    entry.  Returns dict(counts, x, v, qseg, W) with W the field energy of
    every step's field before its kick (n_steps values)."""
    counts = np.array(counts, dtype=np.int32)
    x, v, qseg = _f64(x).copy(), _f64(v).copy(), _f64(qseg).copy()
    W = []
    charge = deposit_seg(nx, L, counts, closed, winding, x, qseg)
    for step in range(n_steps):
        _, E = field(nx, L, charge)
        W.append(field_energy(nx, L, E))
        v = v + dt * qm * gather(nx, L, E, x)
        x = x + dt * v
        if (step + 1) % every == 0:
            counts, x, v, qseg = refine(L, counts, closed, winding, x, v, qseg, l_ref)
        charge = deposit_seg(nx, L, counts, closed, winding, x, qseg)
    return dict(counts=counts, x=x, v=v, qseg=qseg, W=np.array(W))


def refine_c(L, counts, closed, winding, x, v, qseg, l_ref):
    """``refine`` done by the C oracle (orc_refine); same arguments and result."""
    lib = _load()
    counts, closed, winding = _sheets(counts, closed, winding)
    counts = counts.copy()
    n = int(counts.sum())
    cap = 2 * n
    xb = np.zeros(cap); vb = np.zeros(cap); qb = np.zeros(cap)
    xb[:n], vb[:n], qb[:n] = x, v, qseg
    added = lib.orc_refine(float(L), counts.size, _ptr(counts, ctypes.c_int32), _ptr(closed, ctypes.c_uint8),
                           _ptr(winding, ctypes.c_int32), cap, _ptr(xb, ctypes.c_double),
                           _ptr(vb, ctypes.c_double), _ptr(qb, ctypes.c_double), float(l_ref))
    m = n + int(added)
    return counts, xb[:m].copy(), vb[:m].copy(), qb[:m].copy()


def run_refined_each_step(nx, L, dt, counts, closed, winding, x, v, qseg, n_steps, l_ref, qm=1.0,
                          max_growth=4.0, l_split=None):
    """Leapfrog run of box particles with per-particle charges, refined after
    every step in which a particle is longer than l_ref (Sec. 2.6) by passes
    that split every particle longer than l_split (default l_ref) until none
    is, in C (orc_run_refined).  Velocities are v^{-1/2} on entry.  Returns
    dict(counts, x, v, qseg, W, n) with W the field energy of every step's
    field before its kick and n the tracer count after every step.  The
    tracers may grow to max_growth times their number."""
    if l_split is None:
        l_split = l_ref
    lib = _load()
    counts, closed, winding = _sheets(counts, closed, winding)
    counts = counts.copy()
    n0 = int(counts.sum())
    cap = int(max_growth * n0) + 16
    xb = np.zeros(cap); vb = np.zeros(cap); qb = np.zeros(cap)
    xb[:n0], vb[:n0], qb[:n0] = _f64(x), _f64(v), _f64(qseg)
    W = np.zeros(int(n_steps))
    nn = np.zeros(int(n_steps), dtype=np.int64)
    rc = lib.orc_run_refined(int(nx), float(L), float(dt), float(qm), counts.size, _ptr(counts, ctypes.c_int32),
                             _ptr(closed, ctypes.c_uint8), _ptr(winding, ctypes.c_int32), cap,
                             _ptr(xb, ctypes.c_double), _ptr(vb, ctypes.c_double), _ptr(qb, ctypes.c_double),
                             int(n_steps), float(l_ref), float(l_split), _ptr(W, ctypes.c_double),
                             _ptr(nn, ctypes.c_long))
    if rc:
        raise ValueError("the refined tracers outgrew max_growth")
    m = int(counts.sum())
    return dict(counts=counts, x=xb[:m].copy(), v=vb[:m].copy(), qseg=qb[:m].copy(), W=W, n=nn)


def run_problem(p, n_steps=None, record_E=False, order=0):
    """``run`` on a problem from ``paper_1506_07207_gb300.inputs``."""
    return run(p.nx, p.L, p.dt, p.counts, p.closed, p.winding, p.x, p.v, p.w,
               p.n_steps if n_steps is None else n_steps, qm=p.qm,
               half_step_init=p.half_step_init, record_E=record_E, order=order)
