"""GPU parity of the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (derived from the arithmetic):
* per-step deposit and field, on identical input state (the oracle re-deposits
  the GPU's tracers converted to FP64): max |rho_gpu - rho_ref| / max n_ref
  <= 1e-5 and max |E_gpu - E_ref| / (L max n_ref) <= 1e-5.  The FP32 cut
  points of a segment spanning l cells carry ~2e-7 l relative error, the
  fixed-point weights 2^-29 of the largest tracer weight;
* total charge: bit-exact and constant over all steps;
* trajectories: field-energy histories within 1e-3 of the oracle's (relative
  to the history's maximum over the compared window), damping and growth
  rates within 1e-3 relative;
* batching, grid shape and translation by whole cells: bit-identical.
"""
import numpy as np
import pytest

import oracle
from oracle import fits
from paper_1506_07207_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL_STEP = 1e-5


@pytest.fixture(scope="module")
def sic():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1506_07207_gb300 import sic as binding
    return binding


def _oracle_fields(p, x, order=0):
    charge = oracle.deposit(p.nx, p.L, p.counts, p.closed, p.winding, x, p.w, order=order)
    n = charge / (p.L / p.nx)
    rho, E = oracle.field(p.nx, p.L, charge, nodes=(order == 4))   # first order: charge on nodes
    return n, rho, E


def _check_step_parity(sim, p, tol=TOL_STEP, order=0):
    """A-14: deposit + field of the GPU's own state against the oracle."""
    mesh, rho = sim.sic_deposit()
    E = sim.sic_field()
    x, _ = sim.sic_get_state()
    n_ref, rho_ref, E_ref = _oracle_fields(p, x, order)
    gross = np.abs(n_ref).max()
    e_rho = np.abs(rho - rho_ref).max() / gross
    e_E = np.abs(E - E_ref).max() / (p.L * gross)
    assert e_rho <= tol, f"rho error {e_rho:.3e}"
    assert e_E <= tol, f"E error {e_E:.3e}"
    return mesh, e_rho, e_E


def _expected_charge(p, unit):
    sigma = 1.0 / unit
    qh = np.floor(p.w * sigma * 0.5 + 0.5).astype(np.int64)
    total = 0
    base = 0
    for n, c in zip(p.counts, p.closed):
        q = qh[base:base + n]
        total += int(q[:-1].sum() + q[1:].sum())
        if c:
            total += int(q[-1] + q[0])
        base += n
    return total


@pytest.mark.parametrize("seed", [1, 2, 3, 4, 5, 6])
def test_deposit_irregular_sheets(sic, seed):
    """Ragged sheets over several tiles, open and closed, windings -1..1,
    per-tracer weights, zero-length segments, folds and wraps."""
    p = inputs.tiny_problem(seed, n_sheets=6, max_tracers=5000, nx=[64, 100, 389, 8, 750, 2][seed - 1],
                            L=[1.0, 3.0, 2.0, 0.5, 10.0, 1.0][seed - 1])
    sim = sic.Sim.from_problem(p, history_len=8)
    try:
        mesh, _, _ = _check_step_parity(sim, p)
        d = sim.sic_diagnostics()
        assert int(mesh.sum()) == d["charge_fixed"] == _expected_charge(p, d["charge_unit"])
        sim.sic_step(3)
        _check_step_parity(sim, p)
        assert sim.sic_diagnostics()["charge_fixed"] == d["charge_fixed"]
    finally:
        sim.sic_destroy()


def test_single_segments_exact(sic):
    """Dyadic segments: the fixed-point pieces equal the exact overlaps.

    Whole cells inside a segment get floor(q 2^32 / span) units each, so the
    last cell carries the remainder: at most one unit per inside cell, plus
    the FP32 rounding of the first cut (~2e-7 q)."""
    nx, L = 8, 8.0
    cases = [([1.25, 1.75], [0, 1, 0, 0, 0, 0, 0, 0]),
             ([4.0, 1.0], [0, 1 / 3, 1 / 3, 1 / 3, 0, 0, 0, 0]),
             ([2.0, 2.0], [0, 0, 1, 0, 0, 0, 0, 0]),
             ([-0.5, 0.5], [0.5, 0, 0, 0, 0, 0, 0, 0.5]),
             ([0.5, 8.5], [0.125] * 8),     # once around the box
             # 1.25 box lengths: cells 0-2 twice in part (every image counts),
             # the whole-cell interior wraps past the box (the O(1) range path)
             ([0.5, 10.5], [0.15, 0.2, 0.15, 0.1, 0.1, 0.1, 0.1, 0.1]),
             ([13.5, 3.5], [0.1, 0.1, 0.1, 0.15, 0.2, 0.15, 0.1, 0.1])]
    for x, want in cases:
        sim = sic.Sim.sic_create(nx, L, 0.1, [2], [0], [0], x, [0.0, 0.0], [1.0, 1.0],
                                 half_step_init=False)
        try:
            mesh, _ = sim.sic_deposit()
            unit = sim.sic_diagnostics()["charge_unit"]
            got = mesh * unit
            inside = abs(x[1] - x[0]) / (L / nx)
            np.testing.assert_allclose(got, want, rtol=0, atol=(inside + 2) * unit + 2.5e-7)
            assert int(mesh.sum()) * unit == 1.0
        finally:
            sim.sic_destroy()


@pytest.mark.parametrize("maker", ["langmuir", "landau_linear", "landau_nonlinear", "two_stream_config"])
def test_paper_configs_step_parity(sic, maker):
    """Full-size paper configurations, in the launch configuration the bench
    times: initial deposit, then after several fused steps."""
    p = getattr(inputs, maker)()
    sim = sic.Sim.from_problem(p, history_len=64)
    try:
        _check_step_parity(sim, p)
        q0 = sim.sic_diagnostics()["charge_fixed"]
        sim.sic_step(20)
        _check_step_parity(sim, p)
        assert sim.sic_diagnostics()["charge_fixed"] == q0
        hist = sim.sic_history(64)
        assert np.all(hist[:, 3] == q0)
    finally:
        sim.sic_destroy()


def _run_gpu(sic, p, steps):
    sim = sic.Sim.from_problem(p, history_len=steps)
    try:
        sim.sic_step(steps)
        h = sim.sic_history(steps)
        x, v = sim.sic_get_state()
        d = sim.sic_diagnostics()
    finally:
        sim.sic_destroy()
    return h, x, v, d


def test_langmuir_trajectory(sic):
    p = inputs.langmuir()
    h, x, v, d = _run_gpu(sic, p, p.n_steps)
    r = oracle.run_problem(p)
    W, Wr = h[:, 0], r["hist"][:-1, 0]
    assert np.abs(W - Wr).max() <= 1e-3 * Wr.max()
    dxr = (x - r["x"]) / p.L
    assert np.abs(dxr - np.round(dxr)).max() <= 1e-5      # positions modulo the box
    assert np.isclose(d["field_energy"], r["hist"][-1, 0], rtol=1e-3, atol=1e-3 * Wr.max())
    # energy and momentum diagnostics follow the oracle's
    Et, Etr = h[:, 0] + h[:, 1], r["hist"][:-1, 0] + r["hist"][:-1, 1]
    assert np.abs(Et - Etr).max() <= 1e-3 * Etr.max()


def test_energy_sums_through_all_accumulation_paths(sic):
    """A cold plasma (v = 0 at creation, so the finest sum unit, 2^-32) driven
    to several cells per step: an item's KE term soon exceeds what a lane's
    64-bit sum holds (the term goes to the block's 128-bit sum whole) and
    smaller terms overflow it on the way (the lane's sum spills into the
    block's). KE and momentum must still follow the oracle's histories."""
    p = inputs.langmuir(n_tracers=1 << 20, nx=256, amp=1.5, dt=0.1, n_steps=16)
    h, x, v, d = _run_gpu(sic, p, p.n_steps)
    r = oracle.run_problem(p)
    K, Kr = h[:, 1], r["hist"][:-1, 1]
    assert np.abs(v).max() * p.dt / (p.L / p.nx) > 2.0        # several cells per step
    assert np.abs(K - Kr).max() <= 1e-3 * Kr.max()
    P, Pr = h[:, 2], r["hist"][:-1, 2]
    assert np.abs(P - Pr).max() <= 1e-3 * np.sqrt(2.0 * Kr.max() * p.L) + 1e-9


def test_landau_damping_matches_oracle(sic):
    p = inputs.landau_linear()
    h, x, v, d = _run_gpu(sic, p, p.n_steps)
    r = oracle.run_problem(p)
    t = np.arange(p.n_steps) * p.dt
    W, Wr = h[:, 0], r["hist"][:-1, 0]
    win = t <= 30.0
    assert np.abs(W[win] - Wr[win]).max() <= 1e-3 * Wr[win].max()
    g = fits.damping_rate(t, W, 2.0, 30.0)
    gr = fits.damping_rate(t, Wr, 2.0, 30.0)
    assert abs(g / gr - 1) <= 1e-3, (g, gr)


def test_two_stream_growth_matches_oracle(sic):
    p = inputs.two_stream(2.4, 0.1, 0.2, nx=256, n_sheets=64, n_tracers=4096, eps=1e-4, t_end=28.0)
    h, x, v, d = _run_gpu(sic, p, p.n_steps)
    r = oracle.run_problem(p)
    t = np.arange(p.n_steps) * p.dt
    W, Wr = h[:, 0], r["hist"][:-1, 0]
    assert np.abs(W - Wr).max() <= 1e-3 * Wr.max()
    g = fits.growth_rate(t, np.sqrt(W), 10.0, 24.0)
    gr = fits.growth_rate(t, np.sqrt(Wr), 10.0, 24.0)
    assert abs(g / gr - 1) <= 1e-3, (g, gr)


def test_nonlinear_landau_history(sic):
    p = inputs.landau_nonlinear(n_sheets=128, n_tracers=1024)
    h, x, v, d = _run_gpu(sic, p, 400)
    r = oracle.run_problem(p, n_steps=400)
    W, Wr = h[:, 0], r["hist"][:-1, 0]
    pt, py = fits.local_maxima(np.arange(400), W)
    ptr, pyr = fits.local_maxima(np.arange(400), Wr)
    assert len(pt) == len(ptr) and len(pt) >= 3
    np.testing.assert_allclose(py, pyr, rtol=1e-3)


def test_batch_equals_alone_bit_exact(sic):
    probs = [inputs.landau(0.1, 0.4, 128, 32, 3000, t_end=1.0),
             inputs.two_stream(1.5, 0.2, 0.3, 512, 16, 5000, t_end=1.0),
             inputs.tiny_problem(11, n_sheets=5, max_tracers=3000, nx=100, L=2.0),
             inputs.langmuir(nx=64)]
    steps = [12, 5, 9, 16]
    alone = []
    for p, n in zip(probs, steps):
        sim = sic.Sim.from_problem(p, history_len=16)
        sim.sic_step(n)
        alone.append((sim.sic_get_state(), sim.sic_history(16), sim.sic_deposit()[0]))
        sim.sic_destroy()
    sims = [sic.Sim.from_problem(p, history_len=16) for p in probs]
    try:
        sic.sic_step_batch(sims, steps)
        for s, (st, hist, mesh) in zip(sims, alone):
            x, v = s.sic_get_state()
            np.testing.assert_array_equal(x, st[0])
            np.testing.assert_array_equal(v, st[1])
            np.testing.assert_array_equal(s.sic_history(16), hist)
            np.testing.assert_array_equal(s.sic_deposit()[0], mesh)
    finally:
        for s in sims:
            s.sic_destroy()


def test_translation_by_whole_cells_is_exact(sic):
    nx, L = 64, 64.0 / 1024                      # dx = 2^-10, positions dyadic
    rng = np.random.default_rng(3)
    x = np.sort(rng.integers(0, 1 << 16, size=3000)) * 2.0 ** -20
    w = rng.integers(1, 64, size=3000) * 2.0 ** -12
    v = np.zeros_like(x)
    meshes = []
    for shift in (0, 5):
        sim = sic.Sim.sic_create(nx, L, 0.1, [3000], [1], [1], x + shift * L / nx, v, w,
                                 half_step_init=False)
        meshes.append(sim.sic_deposit()[0])
        sim.sic_destroy()
    np.testing.assert_array_equal(meshes[1], np.roll(meshes[0], 5))


def test_strict_mode_reports_long_segment(sic):
    # a segment longer than the box (but inside the position format) at create
    x = np.array([0.0, 0.3, 1.5])
    with pytest.raises(sic.SicError) as e:
        sic.Sim.sic_create(16, 1.0, 0.1, [3], [0], [0], x, np.zeros(3), np.ones(3), strict=True,
                           half_step_init=False)
    assert e.value.code == sic.SIC_ESEGMENT_LONG
    # one that grows past the box while stepping (0.5 + 0.4 per step)
    sim = sic.Sim.sic_create(16, 1.0, 0.1, [2], [0], [0], [0.2, 0.7], [-2.0, 2.0], [1.0, 1.0],
                             strict=True, half_step_init=False, qm=1e-6)
    try:
        sim.sic_step(1)
        sim.sic_sync()
        with pytest.raises(sic.SicError) as e:
            sim.sic_step(1)
            sim.sic_sync()
        assert e.value.code == sic.SIC_ESEGMENT_LONG
    finally:
        sim.sic_destroy()
    # without strict mode the same run deposits every image and keeps charge
    sim = sic.Sim.sic_create(16, 1.0, 0.1, [2], [0], [0], [0.2, 0.7], [-2.0, 2.0], [1.0, 1.0],
                             half_step_init=False, qm=1e-6)
    try:
        sim.sic_step(2)
        d = sim.sic_diagnostics()
        assert 1.2 < d["max_segment"] < 1.5
        assert d["charge_fixed"] * d["charge_unit"] == 1.0
        x, _ = sim.sic_get_state()
        assert abs((x[1] - x[0]) - 1.3) < 1e-6
        # a third step takes it to 1.7 box lengths: past the position format's
        # range (1.5), reported as a range error at the next synchronising call
        with pytest.raises(sic.SicError) as e:
            sim.sic_step(1)
            sim.sic_sync()
        assert e.value.code == sic.SIC_ERANGE
    finally:
        sim.sic_destroy()


def test_position_format_limits_at_create(sic):
    """A segment of 1.5 box lengths or more, or a step of half a box or more,
    is outside the position format: SIC_ERANGE at creation."""
    for x in ([0.0, 1.5], [0.0, -1.6], [0.25, 1.75]):
        with pytest.raises(sic.SicError) as e:
            sic.Sim.sic_create(8, 1.0, 0.1, [2], [0], [0], x, [0.0, 0.0], [1.0, 1.0], half_step_init=False)
        assert e.value.code == sic.SIC_ERANGE
    # the closing segment of a closed sheet counts with its winding
    with pytest.raises(sic.SicError) as e:
        sic.Sim.sic_create(8, 1.0, 0.1, [2], [1], [2], [0.0, 0.25], [0.0, 0.0], [1.0, 1.0], half_step_init=False)
    assert e.value.code == sic.SIC_ERANGE
    with pytest.raises(sic.SicError) as e:
        sic.Sim.sic_create(8, 1.0, 0.1, [2], [0], [0], [0.0, 0.1], [0.0, 5.0], [1.0, 1.0], half_step_init=False)
    assert e.value.code == sic.SIC_ERANGE
    # just inside: 1.4 box lengths, and a step of 0.45 box
    sim = sic.Sim.sic_create(8, 1.0, 0.1, [2], [0], [0], [0.0, 1.4], [0.0, 4.5], [1.0, 1.0], half_step_init=False)
    sim.sic_destroy()


def test_positions_far_from_the_box(sic):
    """Tracers given a thousand boxes away give the same deposit and steps as
    the same tracers inside the box (positions are kept modulo 4 boxes).  The
    positions sit on the format's grid (multiples of L 2^-30, L a power of
    two), so the shifted ones are exact."""
    p = inputs.tiny_problem(41, n_sheets=3, max_tracers=2000, nx=50, L=2.0)
    xq = np.round(p.x / p.L * 2.0 ** 30) * (p.L * 2.0 ** -30)
    runs = []
    for shift in (0.0, 1024.0 * p.L, -3.0 * p.L):
        sim = sic.Sim.sic_create(p.nx, p.L, p.dt, p.counts, p.closed, p.winding, xq + shift, p.v, p.w,
                                 half_step_init=False, history_len=4)
        sim.sic_step(3)
        runs.append((sim.sic_deposit()[0], sim.sic_history(4), sim.sic_get_state()))
        sim.sic_destroy()
    for m, h, (x, v) in runs[1:]:
        np.testing.assert_array_equal(m, runs[0][0])
        np.testing.assert_array_equal(h, runs[0][1])
        np.testing.assert_array_equal(x, runs[0][2][0])
        np.testing.assert_array_equal(v, runs[0][2][1])


def test_grid_shape_does_not_change_results(sic, monkeypatch):
    """Other block counts (down to one block doing everything) give
    bit-identical states, meshes and diagnostic histories."""
    p = inputs.tiny_problem(21, n_sheets=4, max_tracers=9000, nx=300, L=2.0)
    runs = []
    for grid in ["", "7", "1", "33"]:
        monkeypatch.setenv("SIC_GRID", grid)
        sim = sic.Sim.from_problem(p, history_len=8)
        sim.sic_step(6)
        runs.append((sim.sic_get_state(), sim.sic_deposit()[0], sim.sic_history(8)))
        sim.sic_destroy()
    (x0, v0), m0, h0 = runs[0]
    for (x, v), m, h in runs[1:]:
        np.testing.assert_array_equal(x, x0)
        np.testing.assert_array_equal(v, v0)
        np.testing.assert_array_equal(m, m0)
        np.testing.assert_array_equal(h, h0)


def test_persistent_batch_equals_alone(sic):
    probs = [inputs.landau(0.1, 0.4, 128, 32, 3000, t_end=1.0),
             inputs.two_stream(1.5, 0.2, 0.3, 512, 16, 5000, t_end=1.0),
             inputs.langmuir(nx=100),
             inputs.tiny_problem(12, n_sheets=4, max_tracers=2000, nx=64, L=1.0, vscale=0.5)]
    steps = 19      # two graph replays of 8 and three single launches
    alone = []
    for p in probs:
        sim = sic.Sim.from_problem(p, history_len=32)
        sim.sic_step(steps)
        alone.append((sim.sic_get_state(), sim.sic_history(32)))
        sim.sic_destroy()
    sims = [sic.Sim.from_problem(p, history_len=32) for p in probs]
    b = sic.Batch(sims)
    assert b.sic_batch_segments() == sum(p.n_segments for p in probs)
    b.sic_batch_step(steps)
    b.sic_batch_destroy()
    try:
        for s, (st, hist) in zip(sims, alone):
            x, v = s.sic_get_state()
            np.testing.assert_array_equal(x, st[0])
            np.testing.assert_array_equal(v, st[1])
            np.testing.assert_array_equal(s.sic_history(32), hist)
    finally:
        for s in sims:
            s.sic_destroy()


def test_many_small_simulations_batch_equals_alone(sic):
    """Many small simulations beside a few large ones in one launch: blocks
    move between simulations and often arrive when every item is claimed.
    Each simulation still takes exactly its steps, bit-identical to running
    alone."""
    # random per-tracer velocities stretch a sheet's segments; vscale 0.2 keeps
    # them inside the position format's 1.5 box lengths over the 25 steps
    probs = [inputs.tiny_problem(100 + i, n_sheets=2, max_tracers=300, nx=[16, 37, 64][i % 3], L=1.0,
                                 vscale=0.2) for i in range(40)]
    probs += [inputs.landau(0.1, 0.5, 128, 64, 4096, t_end=1.0), inputs.two_stream(1.5, 0.2, 0.3, 256, 32, 8192,
                                                                                     t_end=1.0)]
    steps = 25
    alone = []
    for p in probs:
        sim = sic.Sim.from_problem(p, history_len=4)
        sim.sic_step(steps)
        alone.append(sim.sic_get_state())
        sim.sic_destroy()
    sims = [sic.Sim.from_problem(p, history_len=4) for p in probs]
    try:
        b = sic.Batch(sims)
        b.sic_batch_step(steps)
        b.sic_batch_destroy()
        for s, (x, v) in zip(sims, alone):
            assert s.sic_diagnostics()["step"] == steps
            xg, vg = s.sic_get_state()
            np.testing.assert_array_equal(xg, x)
            np.testing.assert_array_equal(vg, v)
    finally:
        for s in sims:
            s.sic_destroy()


def test_autotuned_batch_equals_plain_batch(sic):
    """The autotuner only changes the schedule: a batch tuned on its first
    steps ends bit-identical to one stepped the same number of times."""
    probs = [inputs.landau(0.1, 0.4, 128, 32, 3000, t_end=1.0),
             inputs.two_stream(1.5, 0.2, 0.3, 512, 16, 5000, t_end=1.0),
             inputs.tiny_problem(31, n_sheets=4, max_tracers=2000, nx=64, L=1.0, vscale=0.2)]
    a = [sic.Sim.from_problem(p, history_len=8) for p in probs]
    b = [sic.Sim.from_problem(p, history_len=8) for p in probs]
    try:
        ba, bb = sic.Batch(a), sic.Batch(b)
        d, st, mn = ba.sic_batch_autotune(2)
        assert d in (1, 2, 4, 8) and st in (0, 1, 2) and mn in (1, 2, 4)
        n_tuned = sic.SIC_AUTOTUNE_CANDIDATES * (2 + 1)
        ba.sic_batch_step(36 - n_tuned)
        bb.sic_batch_step(36)
        ba.sic_batch_destroy()
        bb.sic_batch_destroy()
        for s, t in zip(a, b):
            assert s.sic_diagnostics()["step"] == t.sic_diagnostics()["step"] == 36
            for u, w in zip(s.sic_get_state(), t.sic_get_state()):
                np.testing.assert_array_equal(u, w)
    finally:
        for s in a + b:
            s.sic_destroy()


def test_largest_mesh(sic):
    """nx = SIC_NX_MAX (8192 cells): the largest shared-memory mesh (one block
    per SM, unstaged), deposit and steps against the oracle."""
    p = inputs.tiny_problem(77, n_sheets=4, max_tracers=20000, nx=sic.SIC_NX_MAX, L=3.0, spread=0.05)
    sim = sic.Sim.from_problem(p, history_len=8)
    try:
        mesh, _, _ = _check_step_parity(sim, p)
        q0 = sim.sic_diagnostics()["charge_fixed"]
        sim.sic_step(4)
        _check_step_parity(sim, p)
        assert sim.sic_diagnostics()["charge_fixed"] == q0 == int(mesh.sum())
    finally:
        sim.sic_destroy()


def test_serving_mix_full_size_batch(sic):
    """The bench's launch configuration at full size: the 48 sampled requests
    (282 M segments) resident in one batch.  Every simulation keeps its charge
    to the unit; the largest and a mid-size one end bit-identical to running
    alone; the mid-size one's deposit and field match the oracle."""
    reqs = inputs.serving_mix(n_requests=48, seed=0x5EC5)
    probs = [r.problem() for r in reqs]
    sizes = np.array([p.n_segments for p in probs])
    big = int(np.argmax(sizes))
    mid = int(np.argmin(np.abs(sizes - (1 << 22))))
    steps = 6
    alone = {}
    for k in (big, mid):
        sim = sic.Sim.from_problem(probs[k], history_len=1)
        sim.sic_step(steps)
        alone[k] = sim.sic_deposit()[0]
        sim.sic_destroy()
    sims = [sic.Sim.from_problem(p, history_len=1) for p in probs]
    try:
        q0 = [s.sic_diagnostics()["charge_fixed"] for s in sims]
        b = sic.Batch(sims)
        b.sic_batch_step(steps)
        b.sic_batch_destroy()
        for s, q in zip(sims, q0):
            d = s.sic_diagnostics()
            assert d["step"] == steps and d["charge_fixed"] == q
        for k in (big, mid):
            np.testing.assert_array_equal(sims[k].sic_deposit()[0], alone[k])
        _check_step_parity(sims[mid], probs[mid])
    finally:
        for s in sims:
            s.sic_destroy()
