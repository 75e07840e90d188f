"""Convergence in particles per cell (Sec. 3.3, convergence study of the
Landau problem): a warm plasma of M = 20 horizontal streams on [-4, 4] v_th,
perturbed in velocity (0.026 v_th at the fundamental mode), run for one
plasma period; the error is the mean L1 difference of E_pot(t) from a run
with many more tracers per stream (the oracle's, N = 16384 per stream),
relative to its mean.  Same mesh and time step throughout, so only the tracer
spacing changes.

The paper reads slopes of -2 (box particles) and -4 (piecewise-linear
particles) off its figure for E_pot, twice the order of the density error.
The oracle shows -2.0 for box particles on this set-up and about -3 for the
piecewise-linear ones between 3 and 13 tracers per cell per stream: those
are what the GPU is held to (box: -2 +- 0.3 and within 0.15 of the oracle's
slope; piecewise linear: steeper than -2.5, and 3 times smaller errors than
box particles at the same tracers).  The GPU's errors stay far above its
FP32 floor (about 1e-6 relative) at these sizes."""
import numpy as np
import pytest

import oracle
from paper_1506_07207_gb300 import inputs

pytestmark = pytest.mark.gpu

M, NX, K, V1, DT = 20, 32, 0.5, 0.026, 0.05
NS = [32, 64, 128, 256]


@pytest.fixture(scope="module")
def sic():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1506_07207_gb300 import sic as binding
    return binding


def _problem(N):
    L = 2 * np.pi / K
    vm = -4.0 + 8.0 * (np.arange(M) + 0.5) / M
    dens = np.exp(-0.5 * vm * vm)
    dens /= dens.sum()
    xt = (np.arange(N) + 0.5) * (L / N)
    x = np.tile(xt, M)
    v = np.repeat(vm, N) + V1 * np.cos(K * x)
    w = np.repeat(dens * (L / N), N)
    return inputs.Problem(name=f"landau_v{N}", nx=NX, L=L, dt=DT, n_steps=int(round(2 * np.pi / DT)),
                          counts=np.full(M, N, np.int32), closed=np.ones(M, np.uint8),
                          winding=np.ones(M, np.int32), x_full=x, v_full=v, w_full=w)


def _gpu_W(sic, p, order):
    sim = sic.Sim.from_problem(p, history_len=p.n_steps, order=order)
    try:
        sim.sic_step(p.n_steps)
        return sim.sic_history(p.n_steps)[:, 0]
    finally:
        sim.sic_destroy()


def _errors(W_of, ref):
    return np.array([np.abs(W_of(N) - ref).mean() / ref.mean() for N in NS])


@pytest.mark.parametrize("order", [0, 1])
def test_epot_error_converges_in_particles_per_cell(sic, order):
    ref = oracle.run_problem(_problem(16384), order=order)["hist"][:-1, 0]
    e_gpu = _errors(lambda N: _gpu_W(sic, _problem(N), order), ref)
    e_orc = _errors(lambda N: oracle.run_problem(_problem(N), order=order)["hist"][:-1, 0], ref)
    ppc = M * np.array(NS) / NX
    slope = lambda e: np.polyfit(np.log(ppc[-len(e):]), np.log(e), 1)[0]
    np.testing.assert_allclose(e_gpu, e_orc, rtol=0.25)
    if order == 0:
        assert abs(slope(e_gpu) + 2.0) <= 0.3, slope(e_gpu)
        assert abs(slope(e_gpu) - slope(e_orc)) <= 0.15
    else:
        assert slope(e_gpu[1:]) < -2.5, slope(e_gpu[1:])
        box = _errors(lambda N: _gpu_W(sic, _problem(N), 0),
                      oracle.run_problem(_problem(16384), order=0)["hist"][:-1, 0])
        assert np.all(e_gpu[1:] * 3 < box[1:]), (e_gpu, box)
