"""GPU test of sic_step_batch_static, the stepping call whose launch plan sits
in a fixed device scratch array: on two calls in a row it must leave exactly
the state and diagnostics that sic_step_batch leaves.  Kept in its own file,
collected last, so that it runs both alone in a fresh process and after the
rest of the suite."""
import numpy as np
import pytest

from paper_1506_07207_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sic():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1506_07207_gb300 import sic as binding
    return binding


def _problems():
    return [inputs.landau(0.1, 0.4, 128, 32, 3000, t_end=1.0),
            inputs.two_stream(1.5, 0.2, 0.3, 512, 16, 5000, t_end=1.0),
            inputs.tiny_problem(21, n_sheets=5, max_tracers=3000, nx=100, L=2.0),
            inputs.langmuir(nx=64)]


def _snapshot(sims):
    out = []
    for s in sims:
        x, v = s.sic_get_state()
        d = s.sic_diagnostics()
        out.append((x, v, d["field_energy"], d["kinetic_energy"], d["momentum"], d["charge_fixed"]))
    return out


def test_static_scratch_batch_equals_batch_on_two_calls(sic):
    probs = _problems()
    ref = [sic.Sim.from_problem(p, history_len=16) for p in probs]
    got = [sic.Sim.from_problem(p, history_len=16) for p in probs]
    try:
        for steps in ([7, 3, 12, 5], [4, 9, 0, 11]):
            sic.sic_step_batch(ref, steps)
            sic.sic_step_batch_static(got, steps)
            for a, b in zip(_snapshot(ref), _snapshot(got)):
                np.testing.assert_array_equal(a[0], b[0])
                np.testing.assert_array_equal(a[1], b[1])
                assert a[2:] == b[2:]
            for r, g in zip(ref, got):
                np.testing.assert_array_equal(r.sic_history(16), g.sic_history(16))
    finally:
        for s in ref + got:
            s.sic_destroy()


def test_static_scratch_batch_rejects_too_many(sic):
    p = inputs.langmuir(n_tracers=64, nx=16)
    sims = [sic.Sim.from_problem(p, history_len=1) for _ in range(sic.SIC_STATIC_MAX_SIMS + 1)]
    try:
        with pytest.raises(sic.SicError) as e:
            sic.sic_step_batch_static(sims, [1] * len(sims))
        assert e.value.code == sic.SIC_EINVAL
        x0 = [s.sic_get_state()[0] for s in sims[:3]]
        sic.sic_step_batch_static(sims[:3], [2, 2, 2])   # at the limit or below it works
        assert any(not np.array_equal(a, s.sic_get_state()[0]) for a, s in zip(x0, sims[:3]))
    finally:
        for s in sims:
            s.sic_destroy()
