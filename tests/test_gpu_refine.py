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
