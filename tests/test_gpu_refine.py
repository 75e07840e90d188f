"""GPU parity of the refinement of Sec. 2.6 (sic_refine) against the FP64
oracle's, through the C ABI.

On the same state the decisions (particle length > l_ref) are the same, the
new tracers sit at the centres (fixed point: within a unit L 2^-30) with the mean
velocities (FP32), the total charge is unchanged to the unit, and the deposit
after refinement matches the oracle's with per-particle charges within the
step tolerance (1e-5 of the gross density).  Runs that refine every few steps
follow the oracle's field energy within 1e-3.
"""
import numpy as np
import pytest

import oracle
from paper_1506_07207_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sic():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1506_07207_gb300 import sic as binding
    return binding


def _state_parity(sim, p, counts, qseg, order=0):
    x, _ = sim.sic_get_state()
    mesh, rho = sim.sic_deposit()
    charge = oracle.deposit_seg(p.nx, p.L, counts, p.closed, p.winding, x, qseg, order)
    n_ref = charge / (p.L / p.nx)
    rho_ref, _ = oracle.field(p.nx, p.L, charge)
    assert np.abs(rho - rho_ref).max() <= 1e-5 * np.abs(n_ref).max()
    return mesh


@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("seed", [4, 9])
def test_refine_matches_oracle(sic, seed, order):
    p = inputs.tiny_problem(seed, n_sheets=5, max_tracers=1500, nx=64, L=2.0, spread=0.05)
    sim = sic.Sim.from_problem(p, history_len=4, order=order)
    try:
        sim.sic_step(2)
        x0, v0 = sim.sic_get_state()
        mesh0, _ = sim.sic_deposit()
        q0 = oracle.particle_charges(p.counts, p.closed, p.w)
        l_ref = 0.6 * p.L / p.nx
        added = sim.sic_refine(l_ref)
        c_ref, x_ref, v_ref, q_ref = oracle.refine(p.L, p.counts, p.closed, p.winding, x0, v0, q0, l_ref)
        assert added == int(c_ref.sum() - p.counts.sum()) > 0
        np.testing.assert_array_equal(sim.counts, c_ref)
        x1, v1 = sim.sic_get_state()
        # the new tracer: the lower end plus half the segment, floored to the
        # position unit L 2^-30
        np.testing.assert_allclose(x1, x_ref, rtol=0, atol=p.L * 2.0 ** -29)
        np.testing.assert_allclose(v1, v_ref, rtol=1e-6, atol=1e-7 * np.abs(v0).max())
        mesh1 = _state_parity(sim, p, c_ref, q_ref, order)
        assert mesh1.sum() == mesh0.sum()
        # and it keeps stepping with the new tracers
        sim.sic_step(3)
        assert sim.sic_diagnostics()["charge_fixed"] == int(mesh0.sum())
    finally:
        sim.sic_destroy()


def test_refine_nothing_to_split(sic):
    p = inputs.langmuir(n_tracers=512, nx=64)
    sim = sic.Sim.from_problem(p, history_len=2)
    try:
        assert sim.sic_refine(10 * p.L) == 0
        assert sim.counts.sum() == 512
        with pytest.raises(sic.SicError):
            sim.sic_refine(0.0)
    finally:
        sim.sic_destroy()


def test_refined_two_stream_follows_oracle(sic):
    """Cold two-stream (the set-up of the paper's refinement study, Sec. 2.6:
    10 tracers per cell per stream, 100 cells, dt 0.1, maximum-growth mode),
    refined every 10 steps: field energy and tracer count follow the oracle."""
    nx, ppc = 100, 10
    wb = np.sqrt(0.5)
    v0 = 1.0
    k = (np.sqrt(3.0) / 2.0) * wb / v0
    L = 2 * np.pi / k
    dx = L / nx
    n = nx * ppc
    q = (np.arange(n) + 0.5) * (L / n)
    x1 = q + 0.01 * dx * np.sin(k * q)
    x = np.concatenate([x1, x1])
    v = np.concatenate([np.full(n, v0), np.full(n, -v0)])
    w = np.full(2 * n, 0.5 * L / n)
    counts, closed, winding = [n, n], [1, 1], [1, 1]
    dt, steps, every, l_ref = 0.1, 200, 10, 0.11 * dx
    sim = sic.Sim.sic_create(nx, L, dt, counts, closed, winding, x, v, w, half_step_init=False,
                             history_len=steps)
    W = []
    try:
        for _ in range(steps // every):
            sim.sic_step(every)
            W.append(sim.sic_history(every)[:, 0])
            sim.sic_refine(l_ref)
        W = np.concatenate(W)
        n_gpu = int(sim.counts.sum())
    finally:
        sim.sic_destroy()
    r = oracle.run_refined(nx, L, dt, counts, closed, winding, x, v, oracle.particle_charges(counts, closed, w),
                           steps, l_ref, every)
    assert np.abs(W - r["W"]).max() <= 1e-3 * r["W"].max()
    assert n_gpu > 2.4 * n and abs(n_gpu / r["counts"].sum() - 1) < 0.02


def _stretching(refine_cells=2.0, t_end=30.0):
    """A small two-stream run whose sheets stretch past a couple of cells after
    the instability saturates (refinement due from about t = 15)."""
    p = inputs.two_stream(1.5, 0.05, 0.4, nx=128, n_sheets=16, n_tracers=512, eps=0.05, t_end=t_end)
    p.refine_length = refine_cells * p.L / p.nx
    return p


def test_refinement_hold_is_the_same_alone_and_in_a_batch(sic):
    """A simulation with a refinement length holds after the step that leaves a
    particle longer than it; in a batch it holds at that same step (its own
    decision) while the others go on, and refining it there gives the same
    tracers as alone."""
    p = _stretching()
    others = [inputs.landau(0.1, 0.4, 128, 32, 3000, t_end=40.0), inputs.langmuir(nx=100)]
    alone = sic.Sim.from_problem(p, history_len=8)
    try:
        alone.sic_step(p.n_steps)
        d_alone = alone.sic_diagnostics()
        held_at = d_alone["step"]
        assert 0 < held_at < p.n_steps                 # it held, part way
        x_a, v_a = alone.sic_get_state()
        added_a = alone.sic_refine(p.refine_length)
        assert added_a > 0
        xr_a, vr_a = alone.sic_get_state()
    finally:
        alone.sic_destroy()
    sims = [sic.Sim.from_problem(q, history_len=8) for q in [p] + others]
    try:
        b = sic.Batch(sims)
        b.sic_batch_step(p.n_steps)
        b.sic_batch_destroy()
        assert sims[0].sic_diagnostics()["step"] == held_at
        assert all(s.sic_diagnostics()["step"] == p.n_steps for s in sims[1:])
        x, v = sims[0].sic_get_state()
        np.testing.assert_array_equal(x, x_a)
        np.testing.assert_array_equal(v, v_a)
        assert sims[0].sic_refine(p.refine_length) == added_a
        xr, vr = sims[0].sic_get_state()
        np.testing.assert_array_equal(xr, xr_a)
        np.testing.assert_array_equal(vr, vr_a)
    finally:
        for s in sims:
            s.sic_destroy()


def test_refining_run_follows_the_oracle(sic):
    """sic_run refines whenever a particle outgrows the refinement length
    (Sec. 2.6); the oracle's refined leapfrog (orc_run_refined, pinned to the
    Python rule) does the same.  The field-energy history agrees within 1e-3
    of its maximum and the tracer counts within 2 %."""
    p = _stretching()
    sim = sic.Sim.from_problem(p, history_len=p.n_steps)
    try:
        added = sim.sic_run(p.n_steps)
        h = sim.sic_history(p.n_steps)
        n_gpu = sim.n_tracers
        d = sim.sic_diagnostics()
        q0 = d["charge_fixed"]
    finally:
        sim.sic_destroy()
    assert added > 0 and d["step"] == p.n_steps
    assert np.all(h[:, 3] == q0)
    r0 = oracle.run_problem(p, n_steps=0)             # x^0 and the oracle's v^{-1/2}
    q = oracle.particle_charges(p.counts, p.closed, p.w)
    r = oracle.run_refined_each_step(p.nx, p.L, p.dt, p.counts, p.closed, p.winding, r0["x"], r0["v"], q,
                                     p.n_steps, l_ref=p.refine_length, max_growth=8.0)
    W, Wr = h[:, 0], r["W"]
    assert np.abs(W - Wr).max() <= 1e-3 * Wr.max()
    assert abs(n_gpu / r["n"][-1] - 1) <= 0.02, (n_gpu, r["n"][-1])


def _paper_refinement_setup(ppc=10, n_cells=100, l_cells=1.0):
    """Sec. 2.6 (refinement experiment and its footnote): two cold anti-
    propagating streams at +-v0 with v0 at the cold maximum-growth mode, the
    box its fundamental, 10 tracers per cell per stream, 100 cells,
    dt = 0.1, a sinusoidal position perturbation of 0.01 dx at the fundamental
    mode; the refinement length in cells.  Times are in units of the per-beam
    plasma frequency, as in Sec. 3.2 (maximum growth rate omega_p / 2), so each
    stream has density 1 here."""
    wb = 1.0                          # per-beam plasma frequency: density 1 each
    v0 = 1.0
    k = np.sqrt(3.0) / 2.0 * wb / v0
    L = 2.0 * np.pi / k
    n = ppc * n_cells
    dx = L / n_cells
    q = np.arange(n) * (L / n)
    xt = q + 0.01 * dx * np.sin(k * q)
    p = inputs._horizontal("refine_paper", n_cells, L, 0.1, 300, xt, np.array([v0, -v0]),
                           np.array([1.0, 1.0]), dict(v0=v0, k=k))
    p.refine_length = l_cells * dx
    return p


def test_refinement_factor_of_the_two_stream_setup(sic):
    """Sec. 2.6: in the linear phase (which saturates around t = 17.5) there is
    little refinement; once the phase-space vortex forms the refinement factor
    (tracers now / tracers at the start) grows about exponentially; the
    refinement length sets the onset of that growth but hardly its rate."""
    t_end = 30.0
    runs = {}
    for l_cells in (1.0, 1.0 / 3.0):
        p = _paper_refinement_setup(l_cells=l_cells)
        n0 = p.n_tracers
        sim = sic.Sim.from_problem(p, history_len=1)
        factor = []
        try:
            for _ in range(int(round(t_end / p.dt))):
                sim.sic_run(1)
                factor.append(sim.n_tracers / n0)
        finally:
            sim.sic_destroy()
        runs[l_cells] = np.array(factor)
    t = (np.arange(len(runs[1.0])) + 1) * 0.1
    for l_cells, f in runs.items():
        # little refinement through the linear phase
        assert f[t <= 17.5].max() < 1.05, (l_cells, f[t <= 17.5].max())
        # then growth by an order of magnitude, about exponential: log f is
        # close to a straight line over the stretch where f goes from 2 to 20
        sel = (f >= 2.0) & (f <= 20.0)
        assert sel.sum() >= 15, (l_cells, sel.sum())
        a, b = np.polyfit(t[sel], np.log(f[sel]), 1)
        resid = np.log(f[sel]) - (a * t[sel] + b)
        assert a > 0.2 and np.abs(resid).max() < 0.35, (l_cells, a, np.abs(resid).max())
        runs[l_cells] = (f, a)
    (f1, a1), (f3, a3) = runs[1.0], runs[1.0 / 3.0]
    # the shorter refinement length starts refining earlier ...
    onset = lambda f: t[np.argmax(f >= 2.0)]
    assert onset(f3) < onset(f1)
    # ... at about the same exponential rate
    assert abs(a3 / a1 - 1) < 0.35, (a1, a3)


def test_refinement_stops_at_the_tracer_limit(sic):
    """A refinement that would take the simulation past its tracer limit is
    not done: sic_run returns SIC_ELIMIT at the step that needed it, with the
    state of that step intact (and its charge), so the run's result so far can
    still be read."""
    p = _stretching()
    p.max_tracers = p.n_tracers + 40
    sim = sic.Sim.from_problem(p, history_len=p.n_steps)
    try:
        q0 = sim.sic_diagnostics()["charge_fixed"]
        with pytest.raises(sic.SicError) as e:
            sim.sic_run(p.n_steps)
        assert e.value.code == sic.SIC_ELIMIT
        d = sim.sic_diagnostics()
        assert 0 < d["step"] < p.n_steps and d["charge_fixed"] == q0
        sim._update_counts()
        assert sim.n_tracers <= p.max_tracers
        assert sim.sic_history(p.n_steps).shape[0] == d["step"]
    finally:
        sim.sic_destroy()
