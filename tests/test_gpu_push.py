"""GPU parity of the gather and push (Sec. 2.3: the PIC "gather" by linear
weighting and the "move", kept unchanged for SIC; leapfrog kick-drift, reading
A-4) through the C ABI, element by element.

Tolerances, from the arithmetic:
* against a push computed on the host from the GPU's own field E^0 (sic_field):
  the kick is FP32 with an FP32 field table, so |v - v_ref| <= 8 ulp(FP32) of
  |v| + dt |qm| max|E|; the drift adds dt times that plus the position
  quantum of the fixed-point format (L 2^-30 at most);
* against the FP64 oracle's step on the same initial state: the field itself
  may differ by the per-step bound of reading A-14 (1e-5 L max n), so the
  velocity tolerance grows by dt |qm| times that.
Positions are compared modulo the box length (the library reports each sheet
unwrapped along its tracers, the oracle unwrapped in time).
"""
import numpy as np
import pytest

import oracle
from paper_1506_07207_gb300 import inputs

pytestmark = pytest.mark.gpu

ULP32 = 2.0 ** -24


@pytest.fixture(scope="module")
def sic():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1506_07207_gb300 import sic as binding
    return binding


def wrap_diff(a, b, L):
    """a - b folded into [-L/2, L/2)."""
    d = (np.asarray(a) - np.asarray(b)) / L
    return (d - np.round(d)) * L


def _on_nodes(p, every=7):
    """The problem's positions with every `every`-th tracer moved onto a node
    (the gather then reads one node value exactly), including nodes 0 and nx-1
    and their periodic images."""
    x = p.x.copy()
    dx = p.L / p.nx
    idx = np.arange(0, x.size, every)
    x[idx] = np.round(x[idx] / dx) * dx
    x[1] = 0.0
    x[2] = (p.nx - 1) * dx
    x[3] = -dx                      # node nx-1 one box to the left
    return x


CASES = [  # seed, nx, L, qm, vscale
    (1, 64, 1.0, 1.0, 1.0),
    (2, 100, 3.0, -0.7, 2.0),
    (3, 389, 2.0, 1.3, 0.5),
    (4, 7, 0.5, 1.0, 0.1),
]


@pytest.mark.parametrize("seed,nx,L,qm,vscale", CASES)
def test_one_step_push_elementwise(sic, seed, nx, L, qm, vscale):
    """One fused step from identical state: x and v of every tracer against
    (a) the host push with the GPU's own field and (b) the oracle's step.
    Irregular open and closed sheets, windings -1..1, tracers on nodes, wraps
    across the periodic edge, a non-power-of-two mesh and a negative qm."""
    p = inputs.tiny_problem(seed, n_sheets=5, max_tracers=3000, nx=nx, L=L, dt=0.05, vscale=vscale)
    x0 = _on_nodes(p)
    v0, w = p.v, p.w
    sim = sic.Sim.sic_create(p.nx, p.L, p.dt, p.counts, p.closed, p.winding, x0, v0, w, qm=qm,
                             half_step_init=False, history_len=2)
    try:
        E0 = sim.sic_field()
        sim.sic_step(1)
        x1, v1 = sim.sic_get_state()
    finally:
        sim.sic_destroy()
    dt = p.dt
    # (a) the push alone, with the GPU's field
    ex = oracle.gather(p.nx, p.L, E0, x0)
    v_ref = v0 + dt * qm * ex
    x_ref = x0 + dt * v_ref
    tol_v = 8 * ULP32 * (np.abs(v0).max() + dt * abs(qm) * np.abs(E0).max())
    tol_x = dt * tol_v + p.L * 2.0 ** -29
    assert np.abs(v1 - v_ref).max() <= tol_v
    assert np.abs(wrap_diff(x1, x_ref, p.L)).max() <= tol_x
    # tracers crossed the periodic edge in this step (the wrap is exercised)
    cells0 = np.floor(x0 / (p.L / p.nx))
    assert np.any(np.floor(x_ref / p.L) != np.floor(x0 / p.L)) or np.any(cells0 < 0)
    # (b) against the oracle's own step (its field from its own deposit)
    r = oracle.run(p.nx, p.L, dt, p.counts, p.closed, p.winding, x0, v0, w, 1, qm=qm,
                   half_step_init=False)
    n_max = np.abs(oracle.density(p.nx, p.L, p.counts, p.closed, p.winding, x0, w)).max()
    tol_v2 = tol_v + dt * abs(qm) * 1e-5 * p.L * n_max
    assert np.abs(v1 - r["v"]).max() <= tol_v2
    assert np.abs(wrap_diff(x1, r["x"], p.L)).max() <= dt * tol_v2 + p.L * 2.0 ** -29


def test_sic_push_through_the_abi(sic):
    """sic_push gathers, kicks and drifts with the current field and does not
    re-solve it: two pushes kick with the same E^0; sic_deposit then solves
    the field of the new positions (checked against the oracle, A-14)."""
    p = inputs.tiny_problem(6, n_sheets=4, max_tracers=2500, nx=128, L=2.0, dt=0.1, vscale=1.5)
    qm = 0.8
    x0, v0, w = p.x, p.v, p.w
    sim = sic.Sim.sic_create(p.nx, p.L, p.dt, p.counts, p.closed, p.winding, x0, v0, w, qm=qm,
                             half_step_init=False, history_len=2)
    try:
        E0 = sim.sic_field()
        sim.sic_push()
        x1, v1 = sim.sic_get_state()
        sim.sic_push()
        x2, v2 = sim.sic_get_state()
        np.testing.assert_array_equal(sim.sic_field(), E0)       # no re-solve
        assert sim.sic_diagnostics()["step"] == 0                 # pushes are not steps
        mesh, rho = sim.sic_deposit()
        E2 = sim.sic_field()
    finally:
        sim.sic_destroy()
    dt = p.dt
    tol_v = 8 * ULP32 * (np.abs(v0).max() + 2 * dt * abs(qm) * np.abs(E0).max())
    v1_ref = v0 + dt * qm * oracle.gather(p.nx, p.L, E0, x0)
    assert np.abs(v1 - v1_ref).max() <= tol_v
    assert np.abs(wrap_diff(x1, x0 + dt * v1_ref, p.L)).max() <= dt * tol_v + p.L * 2.0 ** -29
    # the second push starts from the GPU's own state after the first
    v2_ref = v1 + dt * qm * oracle.gather(p.nx, p.L, E0, x1)
    assert np.abs(v2 - v2_ref).max() <= tol_v
    assert np.abs(wrap_diff(x2, x1 + dt * v2_ref, p.L)).max() <= dt * tol_v + p.L * 2.0 ** -29
    # the deposit re-solves the field from x2
    charge = oracle.deposit(p.nx, p.L, p.counts, p.closed, p.winding, x2, w)
    n_ref = charge / (p.L / p.nx)
    rho_ref, E_ref = oracle.field(p.nx, p.L, charge)
    assert np.abs(rho - rho_ref).max() <= 1e-5 * np.abs(n_ref).max()
    assert np.abs(E2 - E_ref).max() <= 1e-5 * p.L * np.abs(n_ref).max()


def test_half_step_start_is_a_half_kick(sic):
    """half_step_init: v^{-1/2} = v^0 - dt/2 qm E^0(x^0) with the field of the
    initial deposit, positions unchanged (reading A-4)."""
    p = inputs.landau(0.2, 0.5, 96, 16, 700, dt=0.1, t_end=0.1)
    qm = 1.0
    sim = sic.Sim.from_problem(p, history_len=1, horizontal=False)
    try:
        E0 = sim.sic_field()
        x, v = sim.sic_get_state()
    finally:
        sim.sic_destroy()
    v_ref = p.v - 0.5 * p.dt * qm * oracle.gather(p.nx, p.L, E0, p.x)
    assert np.abs(v - v_ref).max() <= 8 * ULP32 * (np.abs(p.v).max() + p.dt * np.abs(E0).max())
    assert np.abs(wrap_diff(x, p.x, p.L)).max() <= p.L * 2.0 ** -30
