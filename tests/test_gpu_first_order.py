"""GPU parity of first-order weighting (Sec. 2.4, SIC_DEPOSIT_FIRST) against
the oracle, through the C ABI: each slice of a particle shared between the two
nodes around it by the hat of half-width dx, the field of the node charges by
the trapezoid rule between nodes.

Tolerances as for the box particles (reading A-14): per step on identical
state, node density within 1e-5 of the gross density and E within 1e-5 of
L times it; total charge bit-exact; histories within 1e-3.  Each cell's
zero-order piece is split between its two nodes with one integer rounding
(half a unit), on top of the FP32 cut of the first piece."""
import numpy as np
import pytest

import oracle
from paper_1506_07207_gb300 import inputs

from test_gpu_parity import _check_step_parity, _expected_charge

pytestmark = pytest.mark.gpu
FIRST = 4


@pytest.fixture(scope="module")
def sic():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1506_07207_gb300 import sic as binding
    return binding


@pytest.mark.parametrize("seed", [1, 2, 3, 4, 5])
def test_first_order_irregular_sheets(sic, seed):
    """Ragged open and closed sheets over several work items, windings,
    zero-length particles (point charges: the hat weights of their point),
    particles wrapping the box and crossing many cells, per-tracer weights."""
    p = inputs.tiny_problem(seed, n_sheets=5, max_tracers=3000, nx=[64, 100, 389, 8, 2][seed - 1],
                            L=[1.0, 3.0, 2.0, 0.5, 1.0][seed - 1])
    sim = sic.Sim.from_problem(p, history_len=8, order=FIRST)
    try:
        mesh, _, _ = _check_step_parity(sim, p, order=FIRST)
        d = sim.sic_diagnostics()
        assert int(mesh.sum()) == d["charge_fixed"] == _expected_charge(p, d["charge_unit"])
        sim.sic_step(3)
        _check_step_parity(sim, p, order=FIRST)
        assert sim.sic_diagnostics()["charge_fixed"] == d["charge_fixed"]
    finally:
        sim.sic_destroy()


def test_first_order_single_particles_by_hand(sic):
    """Node charges of single particles (nx = 8, dx = 1, unit charge):
    inside one cell at fractions 1/4 and 3/4, centroid 1/2: half to each node;
    a point at 2.25: 3/4 to node 2, 1/4 to node 3; from 1.5 to 4.5 (three
    cells): pieces 1/6, 1/3, 1/3, 1/6 split by their centroids."""
    nx, L = 8, 8.0
    cases = [([1.25, 1.75], {1: 0.5, 2: 0.5}),
             ([2.25, 2.25], {2: 0.75, 3: 0.25}),
             ([1.5, 4.5], {1: 1 / 6 * 0.25, 2: 1 / 6 * 0.75 + 1 / 3 * 0.5, 3: 1 / 3,
                           4: 1 / 3 * 0.5 + 1 / 6 * 0.75, 5: 1 / 6 * 0.25}),
             ([7.5, 8.5], {7: 0.5 * 0.25, 0: 0.5 * 0.75 + 0.5 * 0.75, 1: 0.5 * 0.25})]
    for x, want in cases:
        sim = sic.Sim.sic_create(nx, L, 0.1, [2], [0], [0], x, [0.0, 0.0], [1.0, 1.0], half_step_init=False,
                                 order=FIRST)
        try:
            mesh, _ = sim.sic_deposit()
            unit = sim.sic_diagnostics()["charge_unit"]
            w = np.zeros(nx)
            for j, c in want.items():
                w[j] = c
            np.testing.assert_allclose(mesh * unit, w, rtol=0, atol=4 * unit + 2.5e-7)
            assert int(mesh.sum()) * unit == 1.0
        finally:
            sim.sic_destroy()


@pytest.mark.parametrize("maker", ["langmuir", "landau_linear", "two_stream_config"])
def test_first_order_paper_configs(sic, maker):
    p = getattr(inputs, maker)()
    sim = sic.Sim.from_problem(p, history_len=32, order=FIRST)
    try:
        _check_step_parity(sim, p, order=FIRST)
        q0 = sim.sic_diagnostics()["charge_fixed"]
        sim.sic_step(20)
        _check_step_parity(sim, p, order=FIRST)
        assert sim.sic_diagnostics()["charge_fixed"] == q0
    finally:
        sim.sic_destroy()


def test_first_order_landau_history_matches_oracle(sic):
    p = inputs.landau(0.05, 0.5, 64, 64, 1024, t_end=15.0)
    sim = sic.Sim.from_problem(p, history_len=p.n_steps, order=FIRST)
    try:
        sim.sic_step(p.n_steps)
        h = sim.sic_history(p.n_steps)
    finally:
        sim.sic_destroy()
    r = oracle.run_problem(p, order=FIRST)
    W, Wr = h[:, 0], r["hist"][:-1, 0]
    assert np.abs(W - Wr).max() <= 1e-3 * Wr.max()


def test_first_order_in_a_mixed_batch_equals_alone(sic):
    probs = [(inputs.landau(0.1, 0.4, 128, 32, 3000, t_end=1.0), FIRST),
             (inputs.two_stream(1.5, 0.2, 0.3, 512, 16, 5000, t_end=1.0), 0),
             (inputs.tiny_problem(14, n_sheets=4, max_tracers=2000, nx=64, L=1.0, vscale=0.3), FIRST)]
    steps = 9
    alone = []
    for p, order in probs:
        sim = sic.Sim.from_problem(p, history_len=16, order=order)
        sim.sic_step(steps)
        alone.append((sim.sic_get_state(), sim.sic_deposit()[0]))
        sim.sic_destroy()
    sims = [sic.Sim.from_problem(p, history_len=16, order=order) for p, order in probs]
    try:
        sic.sic_step_batch(sims, [steps] * len(sims))
        for s, ((x, v), m) in zip(sims, alone):
            xg, vg = s.sic_get_state()
            np.testing.assert_array_equal(xg, x)
            np.testing.assert_array_equal(vg, v)
            np.testing.assert_array_equal(s.sic_deposit()[0], m)
    finally:
        for s in sims:
            s.sic_destroy()
