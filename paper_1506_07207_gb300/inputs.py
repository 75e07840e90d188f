"""Seeded, synthetic initial conditions shaped like the paper's test problems.

This module only builds inputs: tracer positions, velocities and charge weights
of phase-space sheets, and the request mix of the serving benchmark.  It holds
none of the SIC method's arithmetic (no deposit, field solve, gather or push),
so both the CUDA path and the oracle can be fed from it.

Problems (all in units with omega_p = 1 and mean density 1):

* ``langmuir``    cold sheet, x = q + a sin(k q), v = 0 (Sec. 3.1 test, with the
                  perturbation in position instead of velocity).
* ``landau``      M horizontal sheets (Sec. 3.3, "horizontal" set-up and cold
                  start) at velocities on the midpoint grid of [-vmax, vmax], each
                  weighted by the unit Maxwellian; the density perturbation
                  (1 + alpha cos kx) goes into the tracer positions.
* ``two_stream``  two Maxwellian beams at +-v0 (spread sigma), M/2 horizontal
                  sheets each, density perturbation eps in positions (Sec. 3.2).
* ``serving_mix`` a seeded stream of Landau / two-stream requests of differing
                  sizes with Poisson arrival times.

Horizontal sheets are closed loops of winding 1 (x_{N+1} = x_1 + L) whose
tracers all share one position template; ``Problem`` keeps that compact form
(``x_template``, ``v_sheet``, ``w_sheet``) and expands it on demand.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

__all__ = [
    "Problem", "perturbed_positions", "langmuir", "landau", "two_stream",
    "landau_linear", "landau_nonlinear", "two_stream_config", "tiny_problem",
    "SplitMix64", "Request", "serving_mix",
]


@dataclasses.dataclass
class Problem:
    """One simulation's inputs: mesh, time step and sheets of ordered tracers."""

    name: str
    nx: int
    L: float
    dt: float
    n_steps: int
    counts: np.ndarray            # int32 [M] tracers per sheet
    closed: np.ndarray            # uint8 [M] 1 = closed loop
    winding: np.ndarray           # int32 [M] closure offset in box lengths
    qm: float = 1.0
    half_step_init: bool = True
    refine_length: float = 0.0    # Sec. 2.6 refinement length; 0: the run never refines
    refine_split: float = 0.0     # length particles are split to when it refines; 0: refine_length
    max_tracers: int = 0          # refinement limit on the tracer count; 0: the library's
    # full per-tracer arrays (float64), or None when built from the template
    x_full: Optional[np.ndarray] = None
    v_full: Optional[np.ndarray] = None
    w_full: Optional[np.ndarray] = None
    # compact horizontal-sheet form: every sheet shares x_template
    x_template: Optional[np.ndarray] = None
    v_sheet: Optional[np.ndarray] = None
    w_sheet: Optional[np.ndarray] = None   # per-tracer weight of each sheet
    params: dict = dataclasses.field(default_factory=dict)

    @property
    def n_sheets(self) -> int:
        return int(self.counts.size)

    @property
    def n_tracers(self) -> int:
        return int(self.counts.sum())

    @property
    def n_segments(self) -> int:
        return int(self.counts.sum() - (self.closed == 0).sum())

    @property
    def is_horizontal(self) -> bool:
        return self.x_template is not None

    @property
    def x(self) -> np.ndarray:
        if self.x_full is None:
            self.x_full = np.tile(self.x_template, self.n_sheets)
        return self.x_full

    @property
    def v(self) -> np.ndarray:
        if self.v_full is None:
            self.v_full = np.repeat(self.v_sheet, self.x_template.size)
        return self.v_full

    @property
    def w(self) -> np.ndarray:
        if self.w_full is None:
            self.w_full = np.repeat(self.w_sheet, self.x_template.size)
        return self.w_full


def perturbed_positions(n: int, L: float, k: float, alpha: float,
                        offset: float = 0.5) -> np.ndarray:
    """Positions with density proportional to 1 + alpha cos(k x).

    Solves x + (alpha/k) sin(k x) = q_i for q_i = (i + offset) L / n by Newton's
    method in float64 (the map is monotone for |alpha| < 1).
    """
    if not abs(alpha) < 1.0:
        raise ValueError("|alpha| must be < 1")
    q = (np.arange(n, dtype=np.float64) + offset) * (L / n)
    x = q.copy()
    if alpha == 0.0:
        return x
    for _ in range(100):
        g = x + (alpha / k) * np.sin(k * x) - q
        x_new = x - g / (1.0 + alpha * np.cos(k * x))
        if np.max(np.abs(x_new - x)) < 1e-15 * L:
            x = x_new
            break
        x = x_new
    return x


def _horizontal(name, nx, L, dt, n_steps, x_template, v_sheet, dens_sheet, params):
    """Closed horizontal sheets sharing x_template; dens_sheet sums to 1."""
    n = x_template.size
    m = v_sheet.size
    w_sheet = np.asarray(dens_sheet, dtype=np.float64) * (L / n)
    return Problem(name=name, nx=int(nx), L=float(L), dt=float(dt), n_steps=int(n_steps),
                   counts=np.full(m, n, dtype=np.int32),
                   closed=np.ones(m, dtype=np.uint8),
                   winding=np.ones(m, dtype=np.int32),
                   x_template=np.ascontiguousarray(x_template, dtype=np.float64),
                   v_sheet=np.ascontiguousarray(v_sheet, dtype=np.float64),
                   w_sheet=w_sheet, params=params)


def langmuir(n_tracers=4096, nx=64, k=0.5, amp=0.01, dt=0.1, n_steps=500):
    """Cold plasma oscillation: one sheet, x = q + amp sin(k q), v = 0, L = 2 pi / k."""
    L = 2.0 * math.pi / k
    q = np.arange(n_tracers, dtype=np.float64) * (L / n_tracers)
    x = q + amp * np.sin(k * q)
    return _horizontal("langmuir", nx, L, dt, n_steps, x, np.zeros(1), np.ones(1),
                       dict(k=k, amp=amp))


def _midpoints(m: int, lo: float, hi: float) -> np.ndarray:
    return lo + (hi - lo) * (np.arange(m, dtype=np.float64) + 0.5) / m


def landau(alpha, k, nx, n_sheets, n_tracers, dt=0.05, t_end=50.0, vmax=6.0,
           name="landau"):
    """Maxwellian plasma, density (1 + alpha cos k x), M horizontal sheets."""
    L = 2.0 * math.pi / k
    v = _midpoints(n_sheets, -vmax, vmax)
    dens = np.exp(-0.5 * v * v)
    dens /= dens.sum()
    x = perturbed_positions(n_tracers, L, k, alpha)
    n_steps = int(round(t_end / dt))
    return _horizontal(name, nx, L, dt, n_steps, x, v, dens,
                       dict(alpha=alpha, k=k, vmax=vmax))


def two_stream(v0, sigma, k, nx, n_sheets, n_tracers, eps=0.01, dt=0.05,
               t_end=100.0, umax=6.0, name="two_stream"):
    """Two Maxwellian beams at +-v0 (density 1/2 each), n_sheets/2 sheets per beam."""
    if n_sheets % 2:
        raise ValueError("two-stream needs an even sheet count")
    L = 2.0 * math.pi / k
    h = n_sheets // 2
    u = _midpoints(h, -umax, umax)
    g = np.exp(-0.5 * u * u)
    g /= g.sum()
    v = np.concatenate([v0 + sigma * u, -v0 + sigma * u])
    dens = 0.5 * np.concatenate([g, g])
    x = perturbed_positions(n_tracers, L, k, eps)
    n_steps = int(round(t_end / dt))
    return _horizontal(name, nx, L, dt, n_steps, x, v, dens,
                       dict(v0=v0, sigma=sigma, k=k, eps=eps))


def vertical(p: Problem, name=None) -> Problem:
    """The same tracers as the horizontal set-up ``p``, connected the other way
    (Sec. 3.3, phase-space geometry): one open sheet per position, its tracers
    ordered by velocity, each with the weight it has in ``p``.  Every particle
    starts with zero length (all tracers of a sheet share x)."""
    if not p.is_horizontal:
        raise ValueError("needs a horizontal set-up")
    n, m = p.x_template.size, p.v_sheet.size
    x = np.repeat(p.x_template, m)
    v = np.tile(p.v_sheet, n)
    w = np.tile(p.w_sheet, n)
    return Problem(name=name or p.name + "_vertical", nx=p.nx, L=p.L, dt=p.dt, n_steps=p.n_steps,
                   counts=np.full(n, m, dtype=np.int32), closed=np.zeros(n, dtype=np.uint8),
                   winding=np.zeros(n, dtype=np.int32), qm=p.qm, half_step_init=p.half_step_init,
                   x_full=x, v_full=v, w_full=w, params=dict(p.params, connectivity="vertical"))


def landau_linear(**kw):
    """Linear Landau damping: alpha 0.01, k 0.5, Nx 128, 256 x 1024, dt 0.05, t_end 50."""
    args = dict(alpha=0.01, k=0.5, nx=128, n_sheets=256, n_tracers=1024, dt=0.05,
                t_end=50.0, name="landau_linear")
    args.update(kw)
    return landau(**args)


def landau_nonlinear(**kw):
    """Nonlinear Landau damping: alpha 0.5, k 0.5, Nx 512, 1024 x 4096, dt 0.05, t_end 60."""
    args = dict(alpha=0.5, k=0.5, nx=512, n_sheets=1024, n_tracers=4096, dt=0.05,
                t_end=60.0, name="landau_nonlinear")
    args.update(kw)
    return landau(**args)


def two_stream_config(**kw):
    """Two-stream: v0 2.4, sigma 0.1, k 0.2, Nx 1024, 512 x 16384, dt 0.05, t_end 100."""
    args = dict(v0=2.4, sigma=0.1, k=0.2, nx=1024, n_sheets=512, n_tracers=16384,
                eps=0.01, dt=0.05, t_end=100.0, name="two_stream")
    args.update(kw)
    return two_stream(**args)


def tiny_problem(seed: int, n_sheets: int, max_tracers: int, nx: int, L: float = 1.0,
                 dt: float = 0.05, n_steps: int = 4, spread: float = 0.3,
                 open_fraction: float = 0.3, vscale: float = 1.0,
                 allow_degenerate: bool = True) -> Problem:
    """Seeded irregular sheets: ragged counts, open and closed chains, random order.

    Positions wander around a base line so segments overlap, fold, cross the
    periodic edge and sometimes span several cells or the whole box; weights
    differ per tracer.  Used for parity cases beyond the paper's quiet starts.
    """
    rng = SplitMix64(seed)
    counts, closed, winding, xs, vs, ws = [], [], [], [], [], []
    for _ in range(n_sheets):
        n = 2 + int(rng.uniform() * (max_tracers - 1))
        c = 0 if rng.uniform() < open_fraction else 1
        wind = 1 if c else 0
        if c and rng.uniform() < 0.2:
            wind = int(rng.uniform() * 3) - 1       # -1, 0 or 1
        base = rng.uniform() * L
        span = wind * L if wind else (rng.uniform() - 0.5) * L
        t = np.arange(n) / n
        jitter = np.array([(rng.uniform() - 0.5) for _ in range(n)]) * spread * L / max(n, 1) * 4
        x = base + span * t + jitter
        if allow_degenerate and n >= 3 and rng.uniform() < 0.3:
            x[1] = x[2]                              # a zero-length segment
        v = np.array([(rng.uniform() - 0.5) for _ in range(n)]) * vscale
        w = np.array([0.5 + rng.uniform() for _ in range(n)]) * (L / n)
        counts.append(n)
        closed.append(c)
        winding.append(wind if c else 0)
        xs.append(x)
        vs.append(v)
        ws.append(w)
    return Problem(name=f"tiny{seed}", nx=int(nx), L=float(L), dt=float(dt),
                   n_steps=int(n_steps), counts=np.array(counts, dtype=np.int32),
                   closed=np.array(closed, dtype=np.uint8),
                   winding=np.array(winding, dtype=np.int32), half_step_init=False,
                   x_full=np.concatenate(xs), v_full=np.concatenate(vs),
                   w_full=np.concatenate(ws), params=dict(seed=seed))


class SplitMix64:
    """The splitmix64 generator (Steele, Lea & Flood 2014), uniform doubles in [0, 1)."""

    _MASK = (1 << 64) - 1

    def __init__(self, seed: int):
        self.state = seed & self._MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & self._MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & self._MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & self._MASK
        return z ^ (z >> 31)

    def uniform(self) -> float:
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))


@dataclasses.dataclass
class Request:
    """One serving request: a problem recipe plus its arrival time (seconds)."""

    index: int
    arrival: float
    kind: str
    params: dict

    def work(self) -> int:
        p = self.params
        return p["n_sheets"] * p["n_tracers"] * p["n_steps"]

    def problem(self) -> Problem:
        p = dict(self.params)
        steps = p.pop("n_steps")
        dt = p["dt"]
        if self.kind == "landau":
            prob = landau(p["alpha"], p["k"], p["nx"], p["n_sheets"], p["n_tracers"],
                          dt=dt, t_end=steps * dt, name=f"req{self.index}")
        else:
            prob = two_stream(p["v0"], p["sigma"], p["k"], p["nx"], p["n_sheets"],
                              p["n_tracers"], eps=p["eps"], dt=dt, t_end=steps * dt,
                              name=f"req{self.index}")
        prob.n_steps = steps
        # a served run refines once a particle passes half the box length, so
        # it can go on past the point where a particle would outgrow the box
        # (Sec. 3.2, Sec. 2.6), splitting every particle longer than a quarter
        # of the box; refinement may grow it to 4 times its tracers (the count
        # grows about exponentially once the sheets fold, Sec. 2.6)
        prob.refine_length = 0.5 * prob.L
        prob.refine_split = 0.25 * prob.L
        prob.max_tracers = 4 * prob.n_tracers
        return prob


def _pow2(rng: SplitMix64, lo_exp: int, hi_exp: int) -> int:
    return 1 << (lo_exp + int(rng.uniform() * (hi_exp - lo_exp + 1)))


def serving_mix(n_requests=4096, seed=0x5EC5, rate=None, max_sheets_exp=10,
                max_tracers_exp=16, max_nx_exp=11, min_steps=200, max_steps=2000):
    """Seeded request stream: Landau or two-stream runs of differing sizes.

    Landau: alpha log-uniform in [0.001, 0.5], k uniform in [0.3, 0.6].
    Two-stream: v0 uniform in [1, 3], sigma uniform in [0.05, 0.3], k at the
    cold maximum-growth mode k v0 = (sqrt 3 / 2) omega_b with omega_b^2 = 1/2.
    Sheets, tracers per sheet and cells are powers of two, uniform in log2 over
    [32, 2^max_sheets_exp], [512, 2^max_tracers_exp], [64, 2^max_nx_exp];
    steps uniform in [min_steps, max_steps]; dt 0.05.  Arrivals are a Poisson
    process of the given rate (requests/s); rate None puts every arrival at 0.
    """
    rng = SplitMix64(seed)
    out = []
    t = 0.0
    wb = math.sqrt(0.5)
    for i in range(n_requests):
        if rate:
            t += -math.log(1.0 - rng.uniform()) / rate
        kind = "landau" if rng.uniform() < 0.5 else "two_stream"
        m = _pow2(rng, 5, max_sheets_exp)
        n = _pow2(rng, 9, max_tracers_exp)
        nx = _pow2(rng, 6, max_nx_exp)
        steps = min_steps + int(rng.uniform() * (max_steps - min_steps + 1))
        p = dict(n_sheets=m, n_tracers=n, nx=nx, n_steps=steps, dt=0.05)
        if kind == "landau":
            p["alpha"] = math.exp(math.log(0.001) + rng.uniform() * math.log(500.0))
            p["k"] = 0.3 + 0.3 * rng.uniform()
        else:
            p["v0"] = 1.0 + 2.0 * rng.uniform()
            p["sigma"] = 0.05 + 0.25 * rng.uniform()
            p["k"] = (math.sqrt(3.0) / 2.0) * wb / p["v0"]
            p["eps"] = 0.01
        out.append(Request(index=i, arrival=t, kind=kind, params=p))
    return out
