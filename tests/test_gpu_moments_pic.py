"""GPU parity of the moments (sic_moments: zero-order n and j on cells, Sec.
2.3 Eq. rho_sum and Eq. j_sum; first order on nodes, Sec. 2.4), of the PIC
comparison deposits (nearest grid point, cloud in cell) and of vertical-sheet
set-ups (Sec. 3.3), against the FP64 oracle through the C ABI.

Moments are FP64 on both sides on the same state; the GPU's charges are the
fixed-point ones (weights rounded to 2^-29 of the largest), so n agrees within
1e-8 of max |n| and j within 1e-8 of max |n| max |v|.  The PIC deposits are
integer pieces of each tracer's charge: within one unit per piece, compared
with the step tolerance of 1e-5 of the gross density.
"""
import numpy as np
import pytest

import oracle
from paper_1506_07207_gb300 import inputs

from test_gpu_parity import _check_step_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sic():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1506_07207_gb300 import sic as binding
    return binding


def _problems():
    return [inputs.tiny_problem(3, n_sheets=5, max_tracers=3000, nx=64, L=2.0),
            inputs.tiny_problem(8, n_sheets=4, max_tracers=2000, nx=37, L=1.0, vscale=3.0),
            inputs.landau(0.2, 0.5, 64, 32, 2048, t_end=1.0)]


@pytest.mark.parametrize("weighting", [0, 1])
@pytest.mark.parametrize("k", [0, 1, 2])
def test_moments_match_oracle(sic, weighting, k):
    p = _problems()[k]
    sim = sic.Sim.from_problem(p, history_len=4)
    try:
        sim.sic_step(2)
        n, j = sim.sic_moments(weighting)
        x, v = sim.sic_get_state()
    finally:
        sim.sic_destroy()
    n_ref, j_ref = oracle.moments(p.nx, p.L, p.counts, p.closed, p.winding, x, v, p.w, weighting)
    scale_n = np.abs(n_ref).max()
    np.testing.assert_allclose(n, n_ref, rtol=0, atol=1e-8 * scale_n)
    np.testing.assert_allclose(j, j_ref, rtol=0, atol=1e-8 * scale_n * max(np.abs(v).max(), 1e-12))


def test_moments_reject_bad_weighting(sic):
    p = inputs.langmuir(n_tracers=256, nx=16)
    sim = sic.Sim.from_problem(p, history_len=1)
    try:
        with pytest.raises(sic.SicError) as e:
            sim.sic_moments(2)
        assert e.value.code == sic.SIC_EINVAL
    finally:
        sim.sic_destroy()


@pytest.mark.parametrize("scheme", [2, 3])
@pytest.mark.parametrize("k", [0, 2])
def test_pic_deposit_and_steps_match_oracle(sic, scheme, k):
    p = _problems()[k]
    sim = sic.Sim.from_problem(p, history_len=8, order=scheme)
    try:
        mesh, _, _ = _check_step_parity(sim, p, order=scheme)
        q0 = sim.sic_diagnostics()["charge_fixed"]
        assert int(mesh.sum()) == q0
        sim.sic_step(5)
        _check_step_parity(sim, p, order=scheme)
        assert sim.sic_diagnostics()["charge_fixed"] == q0
    finally:
        sim.sic_destroy()


def test_pic_landau_history_matches_oracle(sic):
    p = inputs.landau(0.05, 0.5, 64, 64, 1024, t_end=8.0)
    sim = sic.Sim.from_problem(p, history_len=p.n_steps, order=3)
    try:
        sim.sic_step(p.n_steps)
        h = sim.sic_history(p.n_steps)
    finally:
        sim.sic_destroy()
    r = oracle.run_problem(p, order=3)
    W, Wr = h[:, 0], r["hist"][:-1, 0]
    assert np.abs(W - Wr).max() <= 1e-3 * Wr.max()


@pytest.mark.parametrize("order", [0, 1])
def test_vertical_sheets_match_oracle(sic, order):
    """Open velocity-ordered sheets whose particles all start with zero
    length (every charge in its tracers' cell), then stretch as the
    velocities spread them."""
    p = inputs.vertical(inputs.landau(0.05, 0.5, 64, 24, 160, t_end=6.0))
    sim = sic.Sim.from_problem(p, history_len=p.n_steps, order=order)
    try:
        _check_step_parity(sim, p, order=order)
        sim.sic_step(p.n_steps)
        _check_step_parity(sim, p, order=order)
        h = sim.sic_history(p.n_steps)
    finally:
        sim.sic_destroy()
    r = oracle.run_problem(p, order=order)
    W, Wr = h[:, 0], r["hist"][:-1, 0]
    assert np.abs(W - Wr).max() <= 1e-3 * Wr.max()
