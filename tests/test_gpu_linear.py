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
