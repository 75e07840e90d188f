"""GPU parity of piecewise-linear particles (Sec. 2.5, SIC_DEPOSIT_LINEAR)
against the FP64 oracle's piecewise-linear deposit, through the C ABI.

Same tolerances as the box particles (reading A-14): per step on identical
input state, |rho_gpu - rho_ref| / max n_ref <= 1e-5 and
|E_gpu - E_ref| / (L max n_ref) <= 1e-5; total charge bit-exact; histories
within 1e-3.  The cumulative cuts q (t + kappa t (t - 1)) are FP32, so a
particle whose gradient term kappa is large carries about (1 + |kappa|) 2^-24
relative error per cut; the sheets here keep |kappa| moderate.
"""
import numpy as np
import pytest

import oracle
from paper_1506_07207_gb300 import inputs

from test_gpu_parity import _check_step_parity, _expected_charge

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sic():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1506_07207_gb300 import sic as binding
    return binding


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_linear_deposit_irregular_sheets(sic, seed):
    """Ragged open and closed sheets over several work items, windings, zero
    lengths, folds (no gradient at a fold corner), per-tracer weights."""
    p = inputs.tiny_problem(seed, n_sheets=5, max_tracers=3000, nx=[64, 100, 389, 8][seed - 1],
                            L=[1.0, 3.0, 2.0, 0.5][seed - 1], spread=0.05)
    sim = sic.Sim.from_problem(p, history_len=8, order=1)
    try:
        mesh, _, _ = _check_step_parity(sim, p, order=1)
        d = sim.sic_diagnostics()
        assert int(mesh.sum()) == d["charge_fixed"] == _expected_charge(p, d["charge_unit"])
        sim.sic_step(3)
        _check_step_parity(sim, p, order=1)
        assert sim.sic_diagnostics()["charge_fixed"] == d["charge_fixed"]
    finally:
        sim.sic_destroy()


@pytest.mark.parametrize("maker", ["langmuir", "landau_linear", "two_stream_config"])
def test_linear_paper_configs_step_parity(sic, maker):
    p = getattr(inputs, maker)()
    sim = sic.Sim.from_problem(p, history_len=32, order=1)
    try:
        _check_step_parity(sim, p, order=1)
        q0 = sim.sic_diagnostics()["charge_fixed"]
        sim.sic_step(20)
        _check_step_parity(sim, p, order=1)
        assert sim.sic_diagnostics()["charge_fixed"] == q0
    finally:
        sim.sic_destroy()


def test_linear_differs_from_box_where_the_density_varies(sic):
    """The two orders agree where every particle sits inside one cell and
    differ on a sheet whose particles cross cell edges with a density
    gradient (the Landau start)."""
    p = inputs.landau(0.3, 0.5, 32, 8, 256, t_end=1.0)
    box = sic.Sim.from_problem(p, history_len=1, order=0)
    lin = sic.Sim.from_problem(p, history_len=1, order=1)
    try:
        mb, _ = box.sic_deposit()
        ml, _ = lin.sic_deposit()
        assert mb.sum() == ml.sum()
        assert np.abs(mb - ml).max() > 0
    finally:
        box.sic_destroy()
        lin.sic_destroy()


def test_linear_landau_history_matches_oracle(sic):
    p = inputs.landau(0.05, 0.5, 64, 64, 1024, t_end=10.0)
    sim = sic.Sim.from_problem(p, history_len=p.n_steps, order=1)
    try:
        sim.sic_step(p.n_steps)
        h = sim.sic_history(p.n_steps)
    finally:
        sim.sic_destroy()
    r = oracle.run_problem(p, order=1)
    W, Wr = h[:, 0], r["hist"][:-1, 0]
    assert np.abs(W - Wr).max() <= 1e-3 * Wr.max()


def test_mixed_orders_batch_equals_alone(sic):
    probs = [(inputs.landau(0.1, 0.4, 128, 32, 3000, t_end=1.0), 1),
             (inputs.two_stream(1.5, 0.2, 0.3, 512, 16, 5000, t_end=1.0), 0),
             (inputs.tiny_problem(12, n_sheets=4, max_tracers=2000, nx=64, L=1.0, spread=0.05), 1)]
    steps = 11
    alone = []
    for p, order in probs:
        sim = sic.Sim.from_problem(p, history_len=16, order=order)
        sim.sic_step(steps)
        alone.append(sim.sic_get_state())
        sim.sic_destroy()
    sims = [sic.Sim.from_problem(p, history_len=16, order=order) for p, order in probs]
    try:
        sic.sic_step_batch(sims, [steps] * len(sims))
        for s, (x, v) in zip(sims, alone):
            xg, vg = s.sic_get_state()
            np.testing.assert_array_equal(xg, x)
            np.testing.assert_array_equal(vg, v)
    finally:
        for s in sims:
            s.sic_destroy()


def _kappa_bound_per_cell(p, x, eps):
    """Per-cell bound, in charge units, on the FP32 cut error of
    piecewise-linear particles (Sec. 2.5): a particle of charge q whose density
    is rho0 (1 + 2 kappa (x - c) / l) puts round(q phi(t)) - round(q phi(t'))
    in each cell it touches, phi(t) = t + kappa t (t - 1); FP32 t and phi carry
    about (1 + |kappa|) 2^-24 relative error each, so every touched cell is
    off by at most 2 eps q (1 + |kappa|).  kappa = g l / (2 rho0) with g the
    central difference of the neighbours' rho0 over their centroid distance,
    0 at a fold corner, a zero length or a particle of a box length or more
    (reading A-19).  Closed horizontal sheets only (the Landau and two-stream
    set-ups)."""
    dx = p.L / p.nx
    bound = np.zeros(p.nx)
    base = 0
    for n, wd in zip(p.counts, p.winding):
        xs = x[base:base + n]
        ws = p.w[base:base + n]
        xa = xs
        xb = np.r_[xs[1:], xs[0] + wd * p.L]
        q = 0.5 * (ws + np.roll(ws, -1))
        ln = np.abs(xb - xa)
        c = 0.5 * (xa + xb)
        rho0 = np.where(ln > 0, q / np.where(ln > 0, ln, 1.0), 0.0)
        cp = np.r_[c[-1] - wd * p.L, c[:-1]]
        cn = np.r_[c[1:], c[0] + wd * p.L]
        rp, rn = np.roll(rho0, 1), np.roll(rho0, -1)
        lp, lnn = np.roll(ln, 1), np.roll(ln, -1)
        ordered = ((cp < c) & (c < cn)) | ((cp > c) & (c > cn))
        ok = ordered & (ln > 0) & (lp > 0) & (lnn > 0) & (ln < p.L)
        g = np.where(ok, (rn - rp) / np.where(cn != cp, cn - cp, 1.0), 0.0)
        kappa = np.where(ok & (rho0 > 0), g * ln / (2 * np.where(rho0 > 0, rho0, 1.0)), 0.0)
        err = 2 * eps * q * (1 + np.abs(kappa))
        lo = np.floor(np.minimum(xa, xb) / dx).astype(np.int64)
        hi = np.floor(np.maximum(xa, xb) / dx).astype(np.int64)
        span = np.minimum(hi - lo, p.nx - 1) + 1
        cells = (np.repeat(lo, span) + (np.arange(span.sum()) - np.repeat(np.cumsum(span) - span, span))) % p.nx
        np.add.at(bound, cells, np.repeat(err, span))
        base += n
    return bound


def test_linear_deposit_on_an_evolved_two_stream_state(sic):
    """Piecewise-linear particles on a rolled-up state: a two-stream run
    (Sec. 3.2 set-up, eps 0.05) stepped past saturation, where sheets have
    filamented and neighbouring particle lengths differ a lot.  The deposit of
    the GPU's own state against the oracle's, cell by cell, within the box
    tolerance (1e-5 of the gross density) plus the kappa-dependent FP32 cut
    bound of each cell; total charge exact."""
    p = inputs.two_stream(2.4, 0.1, 0.2, nx=256, n_sheets=64, n_tracers=2048, eps=0.05, t_end=30.0)
    sim = sic.Sim.from_problem(p, history_len=4, order=1)
    try:
        q0 = sim.sic_diagnostics()["charge_fixed"]
        sim.sic_step(p.n_steps)
        x, _ = sim.sic_get_state()
        mesh, _ = sim.sic_deposit()
        unit = sim.sic_diagnostics()["charge_unit"]
        assert int(mesh.sum()) == q0
    finally:
        sim.sic_destroy()
    ref = oracle.deposit(p.nx, p.L, p.counts, p.closed, p.winding, x, p.w, order=1)
    dx = p.L / p.nx
    gross = np.abs(ref).max()
    bound = 1e-5 * gross + _kappa_bound_per_cell(p, x, 8 * 2.0 ** -24) + 4 * unit
    err = np.abs(mesh * unit - ref)
    assert np.all(err <= bound), (err / bound).max()
    # the state is filamented: some particles are many times longer than others
    lens = np.abs(np.diff(x.reshape(len(p.counts), -1), axis=1))
    assert lens.max() > 50 * np.median(lens)
