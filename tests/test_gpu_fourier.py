"""Fourier diagnostics (Sec. 3.2) on the GPU against the FP64 oracle.

* The per-step field energy of the excited mode, recorded by the field solve
  (``mode_k``), against the oracle's mode energy of its own field at every
  step of a two-stream run through the linear growth: the history within
  1e-3 of the largest field energy, its growth rate within 1e-3 of the
  oracle's, and every value at most the total W_E of its step.
* ``sic_spectrum`` of the density and of the node field against the oracle's
  transform of its own deposit of the same tracer positions.
"""
import numpy as np
import pytest

import oracle
from oracle import fits
from paper_1506_07207_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sic():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1506_07207_gb300 import sic as binding
    return binding


def _problem():
    return inputs.two_stream_config(nx=128, n_sheets=32, n_tracers=1024, t_end=17.0)


def test_excited_mode_energy_matches_oracle(sic):
    p = _problem()
    n = p.n_steps
    sim = sic.Sim.from_problem(p, history_len=n, mode_k=1)
    try:
        sim.sic_step(n)
        wk = sim.sic_mode_history(n)
        h = sim.sic_history(n)
    finally:
        sim.sic_destroy()
    assert wk.shape == (n,)
    ref = oracle.run_problem(p, record_E=True)
    wk_ref = np.array([oracle.mode_energy(E, p.L, 1) for E in ref["E_hist"][:n]])
    we_ref = ref["hist"][:n, 0]
    assert np.abs(wk - wk_ref).max() <= 1e-3 * we_ref.max()
    assert np.all(wk <= h[:, 0] * (1 + 1e-5) + 1e-30)
    # the excited mode carries most of the field energy once it has grown
    i14 = int(round(14.0 / p.dt))
    assert wk[i14] > 0.8 * h[i14, 0]
    t = np.arange(n) * p.dt
    g = fits.growth_rate(t, np.sqrt(wk), 12.0, 16.0)
    gr = fits.growth_rate(t, np.sqrt(wk_ref), 12.0, 16.0)
    assert abs(g / gr - 1) <= 1e-3, (g, gr)


def test_mode_history_needs_a_mode(sic):
    p = _problem()
    sim = sic.Sim.from_problem(p, history_len=4)
    try:
        sim.sic_step(2)
        with pytest.raises(sic.SicError):
            sim.sic_mode_history(2)
    finally:
        sim.sic_destroy()
    with pytest.raises(sic.SicError):
        sic.Sim.from_problem(p, history_len=4, mode_k=p.nx // 2 + 1)


@pytest.mark.parametrize("nx", [128, 75])
def test_spectrum_matches_oracle(sic, nx):
    p = inputs.two_stream_config(nx=nx, n_sheets=16, n_tracers=512, t_end=5.0)
    sim = sic.Sim.from_problem(p, history_len=8)
    try:
        sim.sic_step(40)
        x, _ = sim.sic_get_state()
        s_rho = sim.sic_spectrum(0)
        s_E = sim.sic_spectrum(1)
        E_gpu = sim.sic_field()
    finally:
        sim.sic_destroy()
    assert s_rho.shape == (nx // 2 + 1,)
    charge = oracle.deposit(p.nx, p.L, p.counts, p.closed, p.winding, x, p.w)
    rho, E = oracle.field(p.nx, p.L, charge)
    ref_rho = oracle.spectrum(rho)
    ref_E = oracle.spectrum(E)
    np.testing.assert_allclose(s_rho, ref_rho, rtol=0, atol=1e-6 * np.abs(rho).sum())
    np.testing.assert_allclose(s_E, ref_E, rtol=0, atol=1e-6 * np.abs(E).sum())
    # the transform of the device's own field, and the excited mode on top
    np.testing.assert_allclose(s_E, oracle.spectrum(E_gpu), rtol=1e-9, atol=1e-12 * np.abs(E_gpu).sum())
    assert np.argmax(s_rho[1:]) == 0


def test_first_order_mode_energy_matches_oracle(sic):
    p = inputs.two_stream_config(nx=64, n_sheets=16, n_tracers=512, t_end=8.0)
    n = p.n_steps
    sim = sic.Sim.from_problem(p, history_len=n, order=4, mode_k=1)
    try:
        sim.sic_step(n)
        wk = sim.sic_mode_history(n)
    finally:
        sim.sic_destroy()
    ref = oracle.run_problem(p, record_E=True, order=4)
    wk_ref = np.array([oracle.mode_energy(E, p.L, 1) for E in ref["E_hist"][:n]])
    assert np.abs(wk - wk_ref).max() <= 1e-3 * ref["hist"][:n, 0].max()


def test_mode_history_is_the_same_alone_and_in_a_batch(sic):
    p = _problem()
    q = inputs.landau(0.1, 0.5, 128, 32, 1024, t_end=5.0)
    n = 100
    alone = sic.Sim.from_problem(p, history_len=n, mode_k=2)
    a2 = sic.Sim.from_problem(p, history_len=n, mode_k=2)
    other = sic.Sim.from_problem(q, history_len=n, mode_k=1)
    try:
        alone.sic_step(n)
        b = sic.Batch([a2, other])
        b.sic_batch_step(n)
        b.sic_batch_destroy()
        np.testing.assert_array_equal(alone.sic_mode_history(n), a2.sic_mode_history(n))
        np.testing.assert_array_equal(alone.sic_history(n), a2.sic_history(n))
    finally:
        for s in (alone, a2, other):
            s.sic_destroy()
