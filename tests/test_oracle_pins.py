"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Every check here is independent of the oracle's own code: exact rational brute
force over all periodic images, closed forms (inverse Lagrangian map, cosine
sums, leapfrog frequency, kinetic dispersion roots), invariants and symmetries.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import fits, theory
from paper_1506_07207_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_closed_forms.json")


# ---------------------------------------------------------------- deposit ----

def _brute_force_charge(nx, L, counts, closed, winding, x, w):
    """Exact rational charge per cell: every segment clipped against every
    periodic image of every cell (Eq. overlap summed as in Eq. rho_sum)."""
    L = Fraction(L)
    dx = L / nx
    out = [Fraction(0)] * nx
    base = 0
    for n, c, wd in zip(counts, closed, winding):
        segs = [(base + i, base + i + 1, 0) for i in range(n - 1)]
        if c:
            segs.append((base + n - 1, base, int(wd)))
        for i, j, wrap in segs:
            xa = Fraction(float(x[i]))
            xb = Fraction(float(x[j])) + wrap * L
            q = (Fraction(float(w[i])) + Fraction(float(w[j]))) / 2
            a, b = min(xa, xb), max(xa, xb)
            if a == b:
                cell = math.floor(a / dx) % nx
                out[cell] += q
                continue
            m_lo = math.floor(a / L) - 1
            m_hi = math.floor(b / L) + 1
            for cell in range(nx):
                for m in range(m_lo, m_hi + 1):
                    lo = max(a, cell * dx + m * L)
                    hi = min(b, (cell + 1) * dx + m * L)
                    if hi > lo:
                        out[cell] += q * (hi - lo) / (b - a)
        base += n
    return np.array([float(v) for v in out])


def _dyadic(rng, n, scale, denom=64):
    return rng.integers(-4 * denom, 4 * denom, size=n) / denom * scale


@pytest.mark.parametrize("seed", range(12))
def test_deposit_matches_exact_rationals(seed):
    rng = np.random.default_rng(seed)
    nx = int(rng.choice([3, 4, 5, 8, 7]))
    L = float(rng.choice([1.0, 2.0, 8.0, 0.5]))
    n_sheets = int(rng.integers(1, 4))
    counts = rng.integers(2, 6, size=n_sheets).astype(np.int32)
    closed = rng.integers(0, 2, size=n_sheets).astype(np.uint8)
    winding = (rng.integers(-1, 3, size=n_sheets) * closed).astype(np.int32)
    n = int(counts.sum())
    x = _dyadic(rng, n, L / 4)
    # edge-aligned points, a zero-length segment and a multi-box segment
    x[0] = 0.0
    if n > 2:
        x[2] = x[1]
    if n > 3:
        x[3] = x[2] + 2.5 * L
    w = rng.integers(1, 9, size=n) / 8.0
    got = oracle.deposit(nx, L, counts, closed, winding, x, w)
    want = _brute_force_charge(nx, L, counts, closed, winding, x, w)
    np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-13 * max(1.0, np.abs(want).max()))


def test_single_segment_cases():
    nx, L = 4, 4.0              # dx = 1
    one = np.array([2], np.int32)
    op = np.array([0], np.uint8)
    z = np.array([0], np.int32)
    w = np.array([1.0, 1.0])
    # inside one cell
    np.testing.assert_array_equal(oracle.deposit(nx, L, one, op, z, [1.25, 1.75], w), [0, 1, 0, 0])
    # exactly three whole cells, reversed order
    got = oracle.deposit(nx, L, one, op, z, [4.0, 1.0], w)
    np.testing.assert_allclose(got, [0, 1 / 3, 1 / 3, 1 / 3], rtol=1e-15)
    # zero length on an edge: left-closed cells take it
    np.testing.assert_array_equal(oracle.deposit(nx, L, one, op, z, [2.0, 2.0], w), [0, 0, 1, 0])
    # wrapping across x = 0 from below
    got = oracle.deposit(nx, L, one, op, z, [-0.5, 0.5], w)
    np.testing.assert_allclose(got, [0.5, 0, 0, 0.5], rtol=1e-15)
    # twice around the box: every cell gets a quarter
    got = oracle.deposit(nx, L, one, op, z, [0.3, 8.3], w)
    np.testing.assert_allclose(got, [0.25] * 4, rtol=1e-14)


# ------------------------------------------------------- field and gather ----

def test_uniform_sheet_gives_zero_field():
    nx, L, n = 16, 2.0, 64
    x = np.arange(n) * (L / n)
    w = np.full(n, L / n)
    c = oracle.deposit(nx, L, [n], [1], [1], x, w)
    rho, E = oracle.field(nx, L, c)
    assert np.all(c == c[0])
    assert np.all(rho == 0.0) and np.all(E == 0.0)


def test_field_of_cosine_density_closed_form():
    nx, L, A = 64, 3.0, 0.37
    dx = L / nx
    for m in (1, 2, 5, 31):
        th = 2 * np.pi * m / nx
        n = 1.0 + A * np.cos(th * np.arange(nx))
        rho, E = oracle.field(nx, L, n * dx)
        # E'_j = dx A sum_{i<j} cos(th i) = dx A [sin(th(j-1/2)) + sin(th/2)] / (2 sin(th/2));
        # the constant drops out with the mean and sin(th(j-1/2)) has zero mean.
        want = dx * A * np.sin(th * (np.arange(nx) - 0.5)) / (2 * np.sin(th / 2))
        np.testing.assert_allclose(rho, A * np.cos(th * np.arange(nx)), atol=1e-14)
        np.testing.assert_allclose(E, want, atol=1e-14)


def test_monotone_sheet_field_from_inverse_map():
    """One monotone cold sheet: the charge left of x is the inverse of the
    piecewise-linear Lagrangian map, so E at the nodes follows without any
    overlap arithmetic (closed form of Sec. 2.3 for a sheet that never folds)."""
    nx, n, k, amp = 32, 200, 1.0, 0.3
    L = 2 * np.pi / k
    q = np.arange(n) * (L / n)
    x = q + amp * np.sin(k * q) + 0.123
    w = np.full(n, L / n)
    c = oracle.deposit(nx, L, [n], [1], [1], x, w)
    _, E = oracle.field(nx, L, c)
    # cumulative charge as a function of x, extended periodically
    xe = np.concatenate([x - L, x, x + L, [x[0] + 2 * L]])
    le = np.concatenate([q - L, q, q + L, [2 * L]])
    edges = np.arange(nx + 1) * (L / nx)
    lcum = np.interp(edges, xe, le)
    charge = np.diff(lcum)
    np.testing.assert_allclose(c, charge, rtol=1e-12)
    Ep = np.concatenate([[0.0], np.cumsum(charge - L / nx)])[:nx]
    np.testing.assert_allclose(E, Ep - Ep.mean(), atol=1e-12)


def test_gather_linear_weighting():
    nx, L = 8, 4.0
    E = np.array([0.0, 1.0, -2.0, 3.0, 0.5, 0.25, -1.0, 2.0])
    x = np.array([0.0, 0.5, 1.0, 0.25, 3.75, 4.0, -0.25, 8.5])
    # dx = 0.5: node hits, a midpoint, quarter points and the periodic wrap
    want = [0.0, 1.0, -2.0, 0.5, 0.5 * 2.0 + 0.5 * 0.0, 0.0,
            0.5 * 2.0 + 0.5 * 0.0, 1.0]
    np.testing.assert_allclose(oracle.gather(nx, L, E, x), want, rtol=1e-15)


def test_one_leapfrog_step_by_hand():
    """One kick-drift step and its diagnostics row, by hand.  Unequal tracer
    weights make the net force on the tracers non-zero, so the time-centred
    momentum differs from one taken with either velocity alone."""
    nx, n, k = 16, 64, 1.0
    L = 2 * np.pi / k
    q = np.arange(n) * (L / n)
    x0 = q + 0.2 * np.sin(k * q)
    v0 = 0.1 * np.cos(k * q) + 0.05
    w = (L / n) * (1.0 + 0.5 * np.sin(k * q + 1.0))
    dt, qm = 0.3, 1.7

    def field_by_hand(x):
        # the sheet's cumulative charge is linear between tracers (each particle
        # a box, charge (w_i + w_{i+1}) / 2), extended periodically
        qs = 0.5 * (w + np.roll(w, -1))
        c = np.concatenate([[0.0], np.cumsum(qs)[:-1]])
        Q = qs.sum()
        xe = np.concatenate([x - L, x, x + L, [x[0] + 2 * L]])
        le = np.concatenate([c - Q, c, c + Q, [2 * Q]])
        charge = np.diff(np.interp(np.arange(nx + 1) * (L / nx), xe, le))
        Ep = np.concatenate([[0.0], np.cumsum(charge - Q / nx)])[:nx]
        return Ep - Ep.mean()

    E0 = field_by_hand(x0)
    nodes = np.arange(nx + 1) * (L / nx)
    Ex = np.interp(np.mod(x0, L), nodes, np.append(E0, E0[0]))
    v1 = v0 + dt * qm * Ex
    x1 = x0 + dt * v1
    r = oracle.run(nx, L, dt, [n], [1], [1], x0, v0, w, 1, qm=qm, half_step_init=False)
    np.testing.assert_allclose(r["v"], v1, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(r["x"], x1, rtol=1e-12, atol=1e-14)
    # the diagnostics row of the step, time-centred on it (reading A-4):
    # W_E of E^0, KE = 1/2 sum m (v0^2 + v1^2) / 2, P = sum m (v0 + v1) / 2 with
    # m = w / qm, and the total charge; the last row has W_E of E^1
    m = w / qm
    h = r["hist"]
    assert math.isclose(h[0, 0], 0.5 * (L / nx) * np.sum(E0 * E0), rel_tol=1e-12)
    assert math.isclose(h[0, 1], 0.5 * np.sum(m * 0.5 * (v0 * v0 + v1 * v1)), rel_tol=1e-12)
    P = np.sum(m * 0.5 * (v0 + v1))
    assert math.isclose(h[0, 2], P, rel_tol=1e-12)
    assert math.isclose(h[0, 3], w.sum(), rel_tol=1e-14)
    # a momentum or energy taken from one velocity alone misses the row by far
    # more than the 1e-12 it is held to (the self-force nearly cancels, so the
    # momentum margin is about 2e-6 relative)
    for vv in (v0, v1):
        assert abs(np.sum(m * vv) - P) > 1e-7 * abs(P)
        assert abs(0.5 * np.sum(m * vv * vv) - h[0, 1]) > 1e-4 * h[0, 1]
    E1 = field_by_hand(x1)
    np.testing.assert_allclose(r["E"], E1, atol=1e-12)
    assert math.isclose(h[1, 0], 0.5 * (L / nx) * np.sum(E1 * E1), rel_tol=1e-10)
    assert np.isnan(h[1, 1]) and np.isnan(h[1, 2])
    # the half step back at start-up: v^{-1/2} = v^0 - dt/2 qm E^0(x^0)
    r = oracle.run(nx, L, dt, [n], [1], [1], x0, v0, w, 0, qm=qm, half_step_init=True)
    np.testing.assert_allclose(r["v"], v0 - 0.5 * dt * qm * Ex, rtol=1e-12, atol=1e-14)


# -------------------------------------------------------------- invariants ----

def test_invariants_translation_mirror_charge():
    p = inputs.tiny_problem(seed=7, n_sheets=5, max_tracers=40, nx=16, L=2.0)
    dx = p.L / p.nx
    c = oracle.deposit(p.nx, p.L, p.counts, p.closed, p.winding, p.x, p.w)
    rho, E = oracle.field(p.nx, p.L, c)
    # charge conservation: the mesh holds the sum of the segment charges
    qs = 0.0
    base = 0
    for n, cl in zip(p.counts, p.closed):
        ww = p.w[base:base + n]
        qs += 0.5 * (ww[:-1] + ww[1:]).sum() + (0.5 * (ww[-1] + ww[0]) if cl else 0.0)
        base += n
    assert abs(c.sum() - qs) <= 1e-13 * qs
    assert abs(rho.sum()) < 1e-12 * np.abs(rho).max() * p.nx
    assert abs(E.sum()) < 1e-12 * np.abs(E).max() * p.nx
    # translation by exactly one cell (dx is a power of two here) rolls the mesh
    c1 = oracle.deposit(p.nx, p.L, p.counts, p.closed, p.winding, p.x + dx, p.w)
    np.testing.assert_allclose(c1, np.roll(c, 1), rtol=1e-12, atol=1e-14)
    # mirror x -> L - x reverses every sheet's direction (winding -> -winding)
    cm = oracle.deposit(p.nx, p.L, p.counts, p.closed, -p.winding, p.L - p.x, p.w)
    np.testing.assert_allclose(cm, c[::-1], rtol=1e-12, atol=1e-14)
    _, Em = oracle.field(p.nx, p.L, cm)
    np.testing.assert_allclose(Em, -np.roll(E[::-1], 1), rtol=1e-10, atol=1e-13)


# ------------------------------------------------------------ dynamics pins ----

def test_langmuir_closed_forms():
    """Sec. 3.1: a cold sheet oscillates at omega_p (leapfrog: (2/dt) asin(dt/2))
    with field energy (amp^2 L / 4) cos^2(omega t) for x = q + amp sin(k q)."""
    p = inputs.langmuir()
    r = oracle.run_problem(p, record_E=True)
    t = np.arange(p.n_steps + 1) * p.dt
    amp = p.params["amp"]
    assert abs(r["hist"][0, 0] / (amp * amp * p.L / 4) - 1) < 1e-4
    # over the first 10 plasma times the coarse (Nx = 64) grid tracks omega to 1e-3
    m1 = fits.mode(r["E_hist"][:101], 1)
    assert abs(fits.oscillation_omega(t[:101], m1.imag) / theory.leapfrog_omega(p.dt) - 1) < 1e-3
    # total charge is conserved
    assert np.ptp(r["hist"][:, 3]) <= 1e-12 * r["hist"][0, 3]
    # the grid error vanishes as dx -> 0: Nx = 1024 holds omega over 500 steps
    pf = inputs.langmuir(nx=1024)
    rf = oracle.run_problem(pf, record_E=True)
    wf = fits.oscillation_omega(t, fits.mode(rf["E_hist"], 1).imag)
    assert abs(wf / theory.leapfrog_omega(p.dt) - 1) < 2e-4
    et = rf["hist"][:-1, 0] + rf["hist"][:-1, 1]
    assert np.ptp(et) / et.mean() < 0.01


def test_dispersion_function_against_library():
    special = pytest.importorskip("scipy.special")
    pts = [0.3 + 0.2j, 2 - 0.2j, 5 + 1j, 19 + 11j, -3 + 0.01j, 0.5 - 3j, 1e-3 + 1e-3j,
           2.7 - 0.3j, 7 + 0.5j, 30 + 20j]
    for z in pts:
        ref = special.wofz(z)
        assert abs(theory.faddeeva(z) - ref) <= 1e-9 * abs(ref), z


def test_theory_roots_and_paper_closed_forms():
    g = json.load(open(GOLDEN))
    # Landau root for the unit Maxwellian at k = 0.5
    w = theory.landau_root(0.5)
    lit = g["landau_linear_root_k0.5_unit_maxwellian"]
    assert abs(w.real - lit["omega_real"]) < 1e-4 and abs(w.imag - lit["gamma"]) < 1e-4
    eps = theory.kinetic_dielectric(w, 0.5, [(1.0, 0.0, 1.0)])
    assert abs(eps) < 1e-10
    # Sec. 3.2: the cold maximum growth is omega_p/2 (per-beam omega_p) at k v0 = sqrt(3)/2 omega_p
    wb = math.sqrt(0.5)
    kmax = math.sqrt(3) / 2 * wb / 2.4
    assert abs(theory.cold_two_stream_rate(kmax, 2.4) - g["two_stream_max_growth"]["ratio_to_omega_p"] * wb) < 1e-12
    ks = np.linspace(0.01, 0.4, 400)
    assert max(theory.cold_two_stream_rate(k, 2.4) for k in ks) <= wb / 2 + 1e-12
    # Sec. 3.2: stable beyond k = sqrt(2) omega_p / v0
    kc = g["two_stream_instability_threshold"]["sqrt2"] * wb / 2.4
    assert theory.cold_two_stream_rate(kc * 1.001, 2.4) == 0.0
    assert theory.cold_two_stream_rate(kc * 0.999, 2.4) > 0.0
    # a warm beam grows a little slower than the cold one
    gw = theory.warm_two_stream_rate(0.2, 2.4, 0.1)
    gc = theory.cold_two_stream_rate(0.2, 2.4)
    assert 0.995 * gc < gw < gc


@pytest.mark.slow
def test_landau_damping_rate():
    """Sec. 3.3 set-up at the linear Landau configuration: the field energy
    peaks decay at 2 gamma with gamma the kinetic root (within 2 %)."""
    p = inputs.landau_linear()
    r = oracle.run_problem(p)
    t = np.arange(p.n_steps + 1) * p.dt
    g = fits.damping_rate(t, r["hist"][:, 0], 2.0, 30.0)
    assert abs(g / theory.landau_root(0.5).imag - 1) < 0.02
    assert np.ptp(r["hist"][:, 3]) <= 1e-12 * r["hist"][0, 3]


def test_two_stream_growth_rate():
    """Sec. 3.2: the fundamental of a small perturbation grows at the kinetic
    rate of two Maxwellian beams (within 1 %)."""
    p = inputs.two_stream(2.4, 0.1, 0.2, nx=64, n_sheets=32, n_tracers=512, eps=1e-5,
                          t_end=28.0)
    r = oracle.run_problem(p, record_E=True)
    t = np.arange(p.n_steps + 1) * p.dt
    a = np.abs(fits.mode(r["E_hist"], 1))
    g = fits.growth_rate(t, a, 10.0, 28.0)
    assert abs(g / theory.warm_two_stream_rate(0.2, 2.4, 0.1) - 1) < 0.01


# -------------------------------------------- piecewise-linear particles ----
# Sec. 2.5: each particle's density is linear about its centroid, with the
# central-difference gradient over its two neighbours along the sheet.

def test_linear_particles_reproduce_a_linear_density():
    """Tracers at the equal-charge quantiles of rho(x) = alpha + beta x: the
    mean of a linear density over a particle is its value at the centroid, so
    the central difference is exactly beta and every interior particle is
    the true density.  Cells covered by interior particles get the exact
    integral; the box particles of Sec. 2.3 do not."""
    alpha, beta, X, n = 1.0, 0.6, 3.0, 201
    nx, L = 16, 4.0
    dx = L / nx
    total = alpha * X + beta * X * X / 2
    q = total / (n - 1)
    k = np.arange(n)
    x = (-alpha + np.sqrt(alpha * alpha + 2 * beta * k * q)) / beta
    x[-1] = X
    w = np.full(n, q)
    lin = oracle.deposit(nx, L, [n], [0], [0], x, w, order=1)
    box = oracle.deposit(nx, L, [n], [0], [0], x, w, order=0)
    j = np.arange(nx)
    exact = alpha * dx + beta * ((j + 1) ** 2 - j ** 2) * dx * dx / 2
    inner = (j * dx >= x[1]) & ((j + 1) * dx <= x[-2])
    assert inner.sum() >= 8
    np.testing.assert_allclose(lin[inner], exact[inner], rtol=1e-12)
    assert np.abs(box[inner] - exact[inner]).max() > 1e-6
    assert math.isclose(lin.sum(), total, rel_tol=1e-13)


@pytest.mark.parametrize("seed", range(8))
def test_linear_particles_conserve_charge(seed):
    rng = np.random.default_rng(100 + seed)
    nx, L = int(rng.integers(3, 11)), float(rng.choice([1.0, 2.5]))
    counts = [int(c) for c in rng.integers(2, 9, size=3)]
    closed = [int(c) for c in rng.integers(0, 2, size=3)]
    winding = [int(c) for c in rng.integers(-1, 3, size=3)]
    x = _dyadic(rng, sum(counts), L)
    w = rng.integers(1, 9, size=sum(counts)) / 8.0
    lin = oracle.deposit(nx, L, counts, closed, winding, x, w, order=1)
    want = 0.0
    base = 0
    for n, c in zip(counts, closed):
        ws = w[base:base + n]
        want += 0.5 * (ws[:-1] + ws[1:]).sum() + (0.5 * (ws[-1] + ws[0]) if c else 0.0)
        base += n
    assert math.isclose(lin.sum(), want, rel_tol=1e-12)


def test_fold_corner_keeps_the_box_particle():
    """The middle particle's centroid lies beyond both neighbours' (a fold
    corner) and the two others are sheet ends: no gradient anywhere, so the
    deposit is the box deposit.  Without the fold the middle particle gets a
    gradient and the deposits differ."""
    nx, L = 8, 2.0
    w = np.full(4, 0.5)
    folded = np.array([0.1, 0.9, 0.4, 0.2])      # centroids 0.5, 0.65, 0.3
    np.testing.assert_allclose(oracle.deposit(nx, L, [4], [0], [0], folded, w, order=1),
                               oracle.deposit(nx, L, [4], [0], [0], folded, w, order=0), rtol=1e-14, atol=1e-16)
    straight = np.array([0.1, 0.4, 0.9, 1.7])    # centroids 0.25, 0.65, 1.3
    lin = oracle.deposit(nx, L, [4], [0], [0], straight, w, order=1)
    box = oracle.deposit(nx, L, [4], [0], [0], straight, w, order=0)
    assert np.abs(lin - box).max() > 1e-3
    assert math.isclose(lin.sum(), box.sum(), rel_tol=1e-14)


def test_linear_particles_converge_faster():
    """Cell charges of rho = 1 + A cos(2 pi x / L) sampled by N tracers at its
    equal-charge quantiles (one closed sheet): the box particles converge at
    second order, the piecewise-linear ones at third order or better."""
    from scipy.optimize import brentq
    L, nx, A = 1.0, 16, 0.5
    dx = L / nx

    def cdf(x):
        return x + A * L / (2 * np.pi) * np.sin(2 * np.pi * x / L)

    exact = np.diff(cdf(np.arange(nx + 1) * dx))
    Ns = [40, 80, 160, 320, 640]
    err = {0: [], 1: []}
    for N in Ns:
        xs = np.array([brentq(lambda t: cdf(t) - k / N, -1e-9, L + 1e-9) for k in range(N)])
        w = np.full(N, 1.0 / N)
        for order in (0, 1):
            got = oracle.deposit(nx, L, [N], [1], [1], xs, w, order=order)
            err[order].append(np.abs(got - exact).max())
    s0 = np.polyfit(np.log(Ns), np.log(err[0]), 1)[0]
    s1 = np.polyfit(np.log(Ns), np.log(err[1]), 1)[0]
    assert -2.6 < s0 < -1.4, s0
    assert s1 < -2.8, s1
    assert err[1][-1] < 1e-2 * err[0][-1]


def test_linear_particles_run_keeps_charge_and_oscillates():
    """A run with piecewise-linear particles keeps the total charge and still
    oscillates at the leapfrog plasma frequency (Langmuir sheet)."""
    p = inputs.langmuir(n_tracers=512, nx=64)
    r = oracle.run_problem(p, n_steps=80, order=1)
    q = r["hist"][:, 3]
    np.testing.assert_allclose(q, q[0], rtol=1e-13)
    W = r["hist"][:-1, 0]
    t = np.arange(80) * p.dt
    tm, _ = fits.local_maxima(t, W)
    period = 2 * np.mean(np.diff(tm))       # W_E peaks twice per period
    assert abs(2 * np.pi / period / theory.leapfrog_omega(p.dt) - 1) < 2e-3


# --------------------------------------------------- moments (n and j) ----
# Sec. 2.3 (Eq. rho_sum, Eq. j_sum: zero order on cells) and Sec. 2.4 (first
# order: hats on the nodes, velocity linear along each particle).

def test_zero_order_moments_agree_with_the_deposit():
    rng = np.random.default_rng(7)
    nx, L = 12, 2.0
    counts, closed, winding = [40, 17, 9], [1, 0, 1], [1, 0, -1]
    x = _dyadic(rng, 66, L)
    w = rng.integers(1, 9, size=66) / 8.0
    u = 0.375
    n, j = oracle.moments(nx, L, counts, closed, winding, x, np.full(66, u), w, weighting=0)
    np.testing.assert_allclose(n, oracle.deposit(nx, L, counts, closed, winding, x, w) / (L / nx), rtol=1e-13)
    np.testing.assert_allclose(j, u * n, rtol=1e-13, atol=1e-15)


def test_segment_velocity_is_mass_weighted():
    """Sec. 2.3: a particle moves with the mass-weighted mean velocity of its
    two tracers, (m_i v_i + m_j v_j) / (m_i + m_j).  Worked by hand: tracers of
    weights 1 and 3 at velocities 2 and -1 give (2 - 3) / 4 = -1/4 (the plain
    mean would be +1/2); the particle carries (1 + 3) / 2 = 2."""
    nx, L = 4, 4.0                                    # dx = 1
    w, v = [1.0, 3.0], [2.0, -1.0]
    # inside cell 0
    n, j = oracle.moments(nx, L, [2], [0], [0], [0.125, 0.375], v, w, weighting=0)
    np.testing.assert_array_equal(n, [2.0, 0, 0, 0])
    np.testing.assert_array_equal(j, [-0.5, 0, 0, 0])
    # across the edge at x = 1, half in each cell, and reversed in x
    n, j = oracle.moments(nx, L, [2], [0], [0], [1.5, 0.5], v, w, weighting=0)
    np.testing.assert_array_equal(n, [1.0, 1.0, 0, 0])
    np.testing.assert_array_equal(j, [-0.25, -0.25, 0, 0])
    # a zero-length particle is a point charge with the same velocity, and its
    # first-order weights are the hats of its point: 3/4 at node 2, 1/4 at 3
    n, j = oracle.moments(nx, L, [2], [0], [0], [2.25, 2.25], v, w, weighting=1)
    np.testing.assert_allclose(n, [0, 0, 1.5, 0.5], rtol=1e-15)
    np.testing.assert_allclose(j, [0, 0, -0.375, -0.125], rtol=1e-15)


def test_particle_charges_by_hand():
    """q_s = (w_i + w_{i+1}) / 2 (reading A-5); a closed sheet's last entry is
    the closing particle, an open sheet's is 0."""
    q = oracle.particle_charges([3, 2], [1, 0], [1.0, 2.0, 4.0, 8.0, 16.0])
    np.testing.assert_array_equal(q, [1.5, 3.0, 2.5, 12.0, 0.0])


def test_first_order_moments_of_a_cosine_density():
    """CIC weighting of a density 1 + A cos(kx) on the nodes is
    1 + A cos(k X_j) sinc^2(k dx / 2) (the hat's Fourier transform); the
    weights form a partition of unity, so the total is kept."""
    from scipy.optimize import brentq
    L, nx, A, N = 1.0, 16, 0.4, 4000
    k = 2 * np.pi / L
    dx = L / nx

    def cdf(x):
        return x + A / k * np.sin(k * x)

    xs = np.array([brentq(lambda t: cdf(t) - L * i / N, -1e-9, L + 1e-9) for i in range(N)])
    w = np.full(N, L / N)
    n, _ = oracle.moments(nx, L, [N], [1], [1], xs, np.zeros(N), w, weighting=1)
    X = np.arange(nx) * dx
    want = 1 + A * np.cos(k * X) * np.sinc(k * dx / 2 / np.pi) ** 2
    np.testing.assert_allclose(n, want, atol=2e-6)
    assert math.isclose(n.sum() * dx, w.sum(), rel_tol=1e-13)


def test_first_order_current_of_a_linear_velocity_field():
    """A uniform open sheet with v = c x: the velocity interpolated along each
    particle is exactly c x, and the hat average of c x about a node is c X_j,
    so every node whose hat lies inside the sheet gets j = n c X_j."""
    nx, L, c = 20, 5.0, 0.7
    dx = L / nx
    x = np.linspace(0.8, 4.2, 341)
    w = np.full(x.size, 0.01)
    n, j = oracle.moments(nx, L, [x.size], [0], [0], x, c * x, w, weighting=1)
    X = np.arange(nx) * dx
    inside = (X - dx >= x[0]) & (X + dx <= x[-1])
    assert inside.sum() >= 10
    dens = 0.01 / (x[1] - x[0])
    np.testing.assert_allclose(n[inside], dens, rtol=1e-12)
    np.testing.assert_allclose(j[inside], dens * c * X[inside], rtol=1e-12)


# ------------------------------------------------- PIC comparison deposits ----

def test_pic_deposits_by_hand():
    """Point charges: nearest grid point puts a tracer in its own cell; cloud
    in cell shares it between the two cells whose centres bracket it."""
    nx, L = 8, 4.0                                   # dx = 0.5, centres 0.25, 0.75, ...
    x = np.array([0.25, 0.5, 0.6, 3.99, -0.1])
    w = np.array([1.0, 2.0, 4.0, 8.0, 16.0])
    ngp = oracle.deposit(nx, L, [5], [0], [0], x, w, order=2)
    np.testing.assert_array_equal(ngp, [1.0, 6.0, 0, 0, 0, 0, 0, 24.0])
    cic = oracle.deposit(nx, L, [5], [0], [0], x, w, order=3)
    want = np.zeros(nx)
    want[0] += 1.0                                   # on a centre: all of it
    want[0] += 1.0; want[1] += 1.0                   # on an edge: half each
    want[0] += 4.0 * 0.3; want[1] += 4.0 * 0.7       # 0.6 is 0.35 dx past centre 0
    want[7] += 8.0 * (1 - 0.48); want[0] += 8.0 * 0.48   # past the last centre: wraps
    want[7] += 16.0 * 0.7; want[0] += 16.0 * 0.3     # -0.1: 0.3 dx from centre -1 (= 7)
    np.testing.assert_allclose(cic, want, rtol=1e-14, atol=1e-14)
    assert math.isclose(cic.sum(), w.sum(), rel_tol=1e-15)


def test_pic_cloud_in_cell_of_a_uniform_lattice_is_uniform():
    nx, L, per = 16, 2.0, 5
    x = (np.arange(nx * per) + 0.37) * (L / (nx * per))
    w = np.full(x.size, 0.125)
    cic = oracle.deposit(nx, L, [x.size], [1], [1], x, w, order=3)
    np.testing.assert_allclose(cic, cic.mean(), rtol=1e-13)


def test_vertical_sheets_start_as_point_charges():
    """Vertical connectivity (Sec. 3.3): every particle of a velocity-ordered
    sheet starts with zero length, so the deposit puts each particle's whole
    charge in its tracers' cell: the tracer weights, halved at the two ends of
    every open sheet, in the cell of their position."""
    p = inputs.vertical(inputs.landau(0.1, 0.5, 32, 12, 40, t_end=1.0))
    got = oracle.deposit(p.nx, p.L, p.counts, p.closed, p.winding, p.x, p.w)
    w = p.w.reshape(len(p.counts), -1).copy()
    w[:, 0] *= 0.5
    w[:, -1] *= 0.5
    want = np.zeros(p.nx)
    cells = np.floor(p.x.reshape(len(p.counts), -1)[:, 0] / (p.L / p.nx)).astype(int) % p.nx
    for c, row in zip(cells, w):
        want[c] += row.sum()
    np.testing.assert_allclose(got, want, rtol=1e-13)


# ------------------------------------------------------------ refinement ----
# Sec. 2.6: a particle longer than the refinement length gets a new tracer at
# its centre (mean velocity), each half with half the charge.

def _refine_case(seed):
    rng = np.random.default_rng(seed)
    L = 2.0
    counts = [int(c) for c in rng.integers(3, 30, size=4)]
    closed = [1, 0, 1, 0]
    winding = [1, 0, -1, 0]
    x = _dyadic(rng, sum(counts), L, denom=32)
    v = rng.normal(size=sum(counts))
    w = rng.integers(1, 9, size=sum(counts)) / 8.0
    return L, counts, closed, winding, x, v, oracle.particle_charges(counts, closed, w)


@pytest.mark.parametrize("seed", range(6))
def test_refinement_keeps_the_deposit_and_the_charge(seed):
    """Splitting a box particle at its centre into two halves of half the
    charge leaves its density, and so the deposit, unchanged; the inserted
    tracers sit at the centres with the mean velocities."""
    L, counts, closed, winding, x, v, q = _refine_case(seed)
    nx, l_ref = 16, 0.3
    c2, x2, v2, q2 = oracle.refine(L, counts, closed, winding, x, v, q, l_ref)
    before = oracle.deposit_seg(nx, L, counts, closed, winding, x, q)
    after = oracle.deposit_seg(nx, L, c2, closed, winding, x2, q2)
    np.testing.assert_allclose(after, before, rtol=1e-12, atol=1e-13)
    assert math.isclose(q2.sum(), q.sum(), rel_tol=1e-15)
    # one new tracer per particle longer than l_ref
    base, base2 = 0, 0
    for n, n2, c, wd in zip(counts, c2, closed, winding):
        xs = x[base:base + n]
        ends = np.r_[xs[1:], xs[0] + wd * L] if c else xs[1:]
        long_ = np.abs(ends - xs[:len(ends)]) > l_ref
        assert n2 == n + long_.sum()
        # the inserted tracers are the centres of the long particles
        ins = []
        k = base2
        for i in range(n):
            k += 1
            if i < len(ends) and long_[i]:
                ins.append(x2[k])
                k += 1
        np.testing.assert_allclose(ins, 0.5 * (xs[:len(ends)][long_] + ends[long_]), rtol=0, atol=1e-15)
        base += n
        base2 += n2


def test_repeated_refinement_bounds_every_particle():
    L, counts, closed, winding, x, v, q = _refine_case(11)
    l_ref = 0.05
    for _ in range(12):
        counts, x, v, q = oracle.refine(L, counts, closed, winding, x, v, q, l_ref)
    base = 0
    for n, c, wd in zip(counts, closed, winding):
        xs = x[base:base + n]
        ends = np.r_[xs[1:], xs[0] + wd * L] if c else xs[1:]
        assert np.abs(ends - xs[:len(ends)]).max() <= l_ref
        base += n


def test_run_refined_without_refinement_is_the_leapfrog_run():
    """run_refined with no particle longer than l_ref carries the charge on the
    particles but is otherwise the leapfrog loop of orc_run: positions,
    velocities and the field-energy row agree bit for bit."""
    p = inputs.tiny_problem(5, n_sheets=4, max_tracers=60, nx=24, L=2.0, dt=0.05)
    steps = 12
    r = oracle.run(p.nx, p.L, p.dt, p.counts, p.closed, p.winding, p.x, p.v, p.w, steps,
                   half_step_init=False)
    q = oracle.particle_charges(p.counts, p.closed, p.w)
    rr = oracle.run_refined(p.nx, p.L, p.dt, p.counts, p.closed, p.winding, p.x, p.v, q, steps,
                            l_ref=np.inf, every=1)
    np.testing.assert_array_equal(rr["counts"], p.counts)
    np.testing.assert_array_equal(rr["x"], r["x"])
    np.testing.assert_array_equal(rr["v"], r["v"])
    np.testing.assert_array_equal(rr["W"], r["hist"][:-1, 0])


def test_run_refined_splits_without_changing_the_field():
    """With refinement after every 3 steps, the refinement at step 3 leaves the
    deposit unchanged (the halves of a box particle cut at its centre), so the
    field energies of steps 0..3 are those of the unrefined run (to rounding);
    afterwards the new tracers move on their own and the runs part."""
    p = inputs.tiny_problem(8, n_sheets=3, max_tracers=40, nx=32, L=1.0, dt=0.05, spread=0.8)
    q = oracle.particle_charges(p.counts, p.closed, p.w)
    every = 3
    r = oracle.run(p.nx, p.L, p.dt, p.counts, p.closed, p.winding, p.x, p.v, p.w, 8,
                   half_step_init=False)
    rr = oracle.run_refined(p.nx, p.L, p.dt, p.counts, p.closed, p.winding, p.x, p.v, q, 8,
                            l_ref=0.02, every=every)
    assert rr["counts"].sum() > p.counts.sum()
    assert math.isclose(rr["qseg"].sum(), q.sum(), rel_tol=1e-14)
    W, Wr = rr["W"], r["hist"][:-1, 0]
    np.testing.assert_allclose(W[:every + 1], Wr[:every + 1], rtol=1e-11)
    assert np.abs(W[every + 1:] - Wr[every + 1:]).max() > 1e-9 * Wr.max()


def test_linear_particle_a_box_length_long_stays_a_box():
    """Reading A-19: a piecewise-linear particle at least one box length long
    keeps the uniform density of Sec. 2.3 (once a particle outgrows the box the
    run has left the regime the method describes, Sec. 3.2, and a linear
    profile about its centroid would overlap its own periodic image).  Open
    sheet of three particles of lengths 0.1, l, 0.2 on a box of length 1: the
    two end particles have no neighbour on one side and stay boxes; the middle
    one has ordered centroids and unequal neighbour densities, so it gets a
    gradient while l < 1 and none at l = 1."""
    nx, L = 8, 1.0
    w = [0.25, 0.25, 0.25, 0.25]
    for ell, linear in ((0.875, True), (1.0, False), (1.25, False)):
        x = [0.0, 0.125, 0.125 + ell, 0.375 + ell]
        box = oracle.deposit(nx, L, [4], [0], [0], x, w)
        lin = oracle.deposit(nx, L, [4], [0], [0], x, w, order=1)
        if linear:
            assert np.abs(lin - box).max() > 1e-3
        else:
            np.testing.assert_array_equal(lin, box)
        assert math.isclose(lin.sum(), 0.75, rel_tol=1e-15)


# ------------------------------------------------------------------ fits ----

def test_fit_helpers_on_closed_forms():
    """The rate and frequency fits on signals with known answers."""
    t = np.arange(0, 40, 0.05)
    # damping: W = exp(2 gamma t) cos^2(omega t) peaks decay at 2 gamma
    g, w = -0.1533, 1.4157
    W = np.exp(2 * g * t) * np.cos(w * t) ** 2
    assert abs(fits.damping_rate(t, W, 2.0, 30.0) / g - 1) < 1e-3
    # growth: |E| = exp(gamma t)
    assert abs(fits.growth_rate(t, 3.0 * np.exp(0.33488 * t), 5.0, 30.0) - 0.33488) < 1e-12
    # oscillation: cos(omega t + phase)
    assert abs(fits.oscillation_omega(t, np.cos(1.000417 * t + 0.3)) - 1.000417) < 1e-5
    # local maxima of a sampled parabola: refined to the vertex
    tt = np.arange(10.0)
    pt, py = fits.local_maxima(tt, -(tt - 4.3) ** 2 + 2.0)
    assert np.allclose(pt, [4.3]) and np.allclose(py, [2.0])
    # mode: the Fourier coefficient of cos(2 pi m j / nx) is 1/2
    nx = 16
    E = np.cos(2 * np.pi * 3 * np.arange(nx) / nx)[None, :]
    assert abs(fits.mode(E, 3)[0] - 0.5) < 1e-15


@pytest.mark.parametrize("seed", range(6))
def test_c_refinement_equals_the_python_one(seed):
    """orc_refine (C) against oracle.refine (the Sec. 2.6 rule written out in
    Python, pinned above): same counts, tracers, velocities and charges."""
    L, counts, closed, winding, x, v, q = _refine_case(seed)
    for l_ref in (0.05, 0.3, 5.0):
        a = oracle.refine(L, counts, closed, winding, x, v, q, l_ref)
        b = oracle.refine_c(L, counts, closed, winding, x, v, q, l_ref)
        for u, w in zip(a, b):
            np.testing.assert_array_equal(u, w)


def _refined_run_by_hand(p, x, v, q, n_steps, l_ref, l_split):
    """The refinement rule of Sec. 2.6 as a plain Python loop over the oracle's
    pinned pieces: after each kick and drift, if a particle is longer than
    l_ref, split (oracle.refine, pinned above) at l_split until none is."""
    counts = np.array(p.counts, dtype=np.int32)
    x, v, q = x.copy(), v.copy(), q.copy()
    W = []
    charge = oracle.deposit_seg(p.nx, p.L, counts, p.closed, p.winding, x, q)
    for _ in range(n_steps):
        _, E = oracle.field(p.nx, p.L, charge)
        W.append(oracle.field_energy(p.nx, p.L, E))
        v = v + p.dt * 1.0 * oracle.gather(p.nx, p.L, E, x)
        x = x + p.dt * v
        base, longest = 0, 0.0
        for n, c, wd in zip(counts, p.closed, p.winding):
            xs = x[base:base + n]
            ends = np.r_[xs[1:], xs[0] + wd * p.L] if c else xs[1:]
            longest = max(longest, np.abs(ends - xs[:len(ends)]).max())
            base += n
        if longest > l_ref:
            while True:
                c2, x, v, q = oracle.refine(p.L, counts, p.closed, p.winding, x, v, q, l_split)
                added = c2.sum() - counts.sum()
                counts = c2
                if added == 0:
                    break
        charge = oracle.deposit_seg(p.nx, p.L, counts, p.closed, p.winding, x, q)
    return counts, x, v, q, np.array(W)


def test_refined_run_in_c_reduces_to_the_known_loops():
    """orc_run_refined with no particle longer than l_ref is orc_run bit for
    bit; with refinement it equals the rule written out as a Python loop over
    the pinned oracle pieces, bit for bit, with the split length equal to the
    hold length and with a shorter one (splitting ahead)."""
    p = inputs.tiny_problem(5, n_sheets=4, max_tracers=60, nx=24, L=2.0, dt=0.05)
    q = oracle.particle_charges(p.counts, p.closed, p.w)
    steps = 12
    r = oracle.run(p.nx, p.L, p.dt, p.counts, p.closed, p.winding, p.x, p.v, p.w, steps, half_step_init=False)
    c = oracle.run_refined_each_step(p.nx, p.L, p.dt, p.counts, p.closed, p.winding, p.x, p.v, q, steps,
                                     l_ref=np.inf)
    np.testing.assert_array_equal(c["x"], r["x"])
    np.testing.assert_array_equal(c["v"], r["v"])
    np.testing.assert_array_equal(c["W"], r["hist"][:-1, 0])
    p = inputs.tiny_problem(8, n_sheets=3, max_tracers=40, nx=32, L=1.0, dt=0.05, spread=0.8)
    q = oracle.particle_charges(p.counts, p.closed, p.w)
    for l_ref, l_split in ((0.1, 0.1), (0.1, 0.03)):
        hand = _refined_run_by_hand(p, p.x, p.v, q, 10, l_ref, l_split)
        c = oracle.run_refined_each_step(p.nx, p.L, p.dt, p.counts, p.closed, p.winding, p.x, p.v, q, 10,
                                         l_ref=l_ref, l_split=l_split, max_growth=64.0)
        assert c["counts"].sum() > 2 * p.counts.sum()
        for got, want in zip((c["counts"], c["x"], c["v"], c["qseg"], c["W"]), hand):
            np.testing.assert_array_equal(got, want)
        assert c["n"][-1] == c["counts"].sum() and np.all(np.diff(c["n"]) >= 0)


# ------------------------------------------- first-order weighting (NEXT-3) ----
# Sec. 2.4: each slice of a particle shared between the two nodes around it by
# the hat of half-width dx; the field of the node charges by the trapezoid rule.

def test_node_field_by_hand():
    """Trapezoid integration between nodes, worked by hand: one unit of extra
    charge on node 0 of four nodes (dx = 1, mean 1/4 per node).  rho =
    (3/4, -1/4, -1/4, -1/4); E' = 0, (3/4 - 1/4)/2, that - 1/4, that - 1/4 =
    0, 1/4, 0, -1/4 (mean 0)."""
    rho, E = oracle.field(4, 4.0, [1.0, 0.0, 0.0, 0.0], nodes=True)
    np.testing.assert_allclose(rho, [0.75, -0.25, -0.25, -0.25], rtol=0, atol=1e-15)
    np.testing.assert_allclose(E, [0.0, 0.25, 0.0, -0.25], rtol=0, atol=1e-15)


def test_first_order_field_of_a_cosine_density():
    """A density 1 + A cos(kx) weighted to the nodes by the hat gives node
    charge dx (1 + A s^2 cos(k X_j)), s = sinc(k dx / 2); the trapezoid rule
    integrates A s^2 cos(k X) between nodes to E_j = (A / k) s^2 (h / tan h)
    sin(k X_j), h = k dx / 2 (sum the differences of sines).  The tracers
    resolve the density to O(1/N^2)."""
    from scipy.optimize import brentq
    L, nx, A, N = 1.0, 16, 0.4, 4000
    k = 2 * np.pi / L
    dx = L / nx

    def cdf(x):
        return x + A / k * np.sin(k * x)

    xs = np.array([brentq(lambda t: cdf(t) - L * i / N, -1e-9, L + 1e-9) for i in range(N)])
    w = np.full(N, L / N)
    charge = oracle.deposit(nx, L, [N], [1], [1], xs, w, order=4)
    assert math.isclose(charge.sum(), w.sum(), rel_tol=1e-13)
    X = np.arange(nx) * dx
    s2 = np.sinc(k * dx / 2 / np.pi) ** 2
    np.testing.assert_allclose(charge / dx, 1 + A * s2 * np.cos(k * X), atol=2e-6)
    _, E = oracle.field(nx, L, charge, nodes=True)
    h = k * dx / 2
    np.testing.assert_allclose(E, (A / k) * s2 * (h / np.tan(h)) * np.sin(k * X), atol=2e-7)


def test_first_order_uniform_sheet_and_charge():
    """A closed sheet of evenly spaced tracers puts the same charge on every
    node (zero field); on random sheets the node charges sum to the charge."""
    nx, L, n = 8, 2.0, 64
    x = (np.arange(n) + 0.3) * (L / n)
    c = oracle.deposit(nx, L, [n], [1], [1], x, np.full(n, L / n), order=4)
    np.testing.assert_allclose(c, L / nx, rtol=1e-13)
    _, E = oracle.field(nx, L, c, nodes=True)
    assert np.abs(E).max() < 1e-13
    p = inputs.tiny_problem(9, n_sheets=5, max_tracers=50, nx=12, L=2.0)
    c = oracle.deposit(p.nx, p.L, p.counts, p.closed, p.winding, p.x, p.w, order=4)
    q = oracle.particle_charges(p.counts, p.closed, p.w)
    assert math.isclose(c.sum(), q.sum(), rel_tol=1e-13)


def test_first_order_run_keeps_charge_and_oscillates():
    """A Langmuir run with first-order weighting: total charge constant and
    the leapfrog plasma frequency (as for the other deposits)."""
    p = inputs.langmuir(nx=128)
    r = oracle.run_problem(p, record_E=True, order=4)
    assert np.ptp(r["hist"][:, 3]) <= 1e-12 * r["hist"][0, 3]
    t = np.arange(p.n_steps + 1) * p.dt
    w = fits.oscillation_omega(t, fits.mode(r["E_hist"], 1).imag)
    assert abs(w / theory.leapfrog_omega(p.dt) - 1) < 2e-3


# ---- Fourier diagnostics (Sec. 3.2: the energy in the excited mode, the
# transform of the charge density)

@pytest.mark.parametrize("nx", [16, 17, 64])
def test_spectrum_matches_the_library_fft(nx):
    rng = np.random.default_rng(nx)
    X = rng.normal(size=nx)
    np.testing.assert_allclose(oracle.spectrum(X), np.abs(np.fft.rfft(X)), rtol=1e-12, atol=1e-12)
    # the sign of the phase: a sine has X^_1 = -i nx / 2
    j = np.arange(nx)
    z = oracle.dft(np.sin(2 * np.pi * j / nx), 1)
    assert abs(z - (-0.5j * nx)) < 1e-10 * nx


@pytest.mark.parametrize("nx", [16, 17, 64])
def test_mode_energies_add_up_to_the_field_energy(nx):
    rng = np.random.default_rng(100 + nx)
    E = rng.normal(size=nx)
    E -= E.mean()
    L = 3.7
    total = sum(oracle.mode_energy(E, L, k) for k in range(1, nx // 2 + 1))
    assert abs(total - oracle.field_energy(nx, L, E)) <= 1e-12 * oracle.field_energy(nx, L, E)


def test_single_cosine_mode_energy():
    nx, L, A, m = 32, 2.0, 0.3, 3
    j = np.arange(nx)
    E = A * np.cos(2 * np.pi * m * j / nx + 0.4)
    # W_E = 1/2 A^2 (L / 2), all of it in mode m
    assert abs(oracle.mode_energy(E, L, m) - A * A * L / 4) < 1e-14
    assert abs(oracle.field_energy(nx, L, E) - A * A * L / 4) < 1e-14
    for k in range(1, nx // 2 + 1):
        if k != m:
            assert oracle.mode_energy(E, L, k) < 1e-28
    # the Nyquist mode alone: E_j = A (-1)^j carries A^2 L / 2
    En = A * (-1.0) ** j
    assert abs(oracle.mode_energy(En, L, nx // 2) - A * A * L / 2) < 1e-14
