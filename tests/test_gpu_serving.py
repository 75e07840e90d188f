"""GPU tests of the request server: continuous batching gives every request
the same bits as running it alone, admission respects the memory budget,
requests that arrive mid-run join the batch, oversize requests are refused."""
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


def _mix(n, seed=7):
    reqs = inputs.serving_mix(n_requests=n, seed=seed, max_sheets_exp=7, max_tracers_exp=12,
                              max_nx_exp=10, min_steps=20, max_steps=90)
    return [r.problem() for r in reqs]


def _alone(sic, p):
    sim = sic.Sim.from_problem(p, history_len=1)
    try:
        sim.sic_step(p.n_steps)
        d = sim.sic_diagnostics()
    finally:
        sim.sic_destroy()
    return d


def _key(d):
    return (d["field_energy"], d["kinetic_energy"], d["momentum"], d["charge_fixed"])


def test_batched_results_equal_alone(sic):
    probs = _mix(10)
    srv = sic.Server(hbm_budget=8 << 30, max_active=4, chunk_steps=16)
    ids = [srv.sic_server_submit_horizontal(p) for p in probs]
    got = {}
    while srv.sic_server_tick() > 0:
        for r in srv.sic_server_results():
            got[r["id"]] = r
    for r in srv.sic_server_results():
        got[r["id"]] = r
    srv.sic_server_destroy()
    assert sorted(got) == sorted(ids)
    for rid, p in zip(ids, probs):
        r = got[rid]
        assert r["status"] == 0 and r["steps"] == p.n_steps
        d = _alone(sic, p)
        assert (r["field_energy"], r["kinetic_energy"], r["momentum"], r["charge_fixed"]) == _key(d)
        assert r["segment_updates"] == p.n_segments * p.n_steps


def test_plain_mode_matches_batched(sic):
    probs = _mix(5, seed=11)
    out = []
    for plain in (True, False):
        srv = sic.Server(hbm_budget=8 << 30, max_active=8, chunk_steps=7, plain=plain)
        ids = [srv.sic_server_submit_horizontal(p) for p in probs]
        got = {}
        while srv.sic_server_tick() > 0:
            pass
        for r in srv.sic_server_results():
            got[r["id"]] = r
        srv.sic_server_destroy()
        out.append([(got[i]["field_energy"], got[i]["kinetic_energy"], got[i]["momentum"]) for i in ids])
    assert out[0] == out[1]


def test_budget_limits_admission(sic):
    probs = _mix(8, seed=3)
    sizes = []
    for p in probs:      # device bytes per request, from a solo run of the server
        srv = sic.Server(hbm_budget=8 << 30, max_active=1, chunk_steps=1000)
        srv.sic_server_submit_horizontal(p, n_steps=0)
        srv.sic_server_tick()
        sizes.append(srv.sic_server_stats()["bytes_peak"])
        srv.sic_server_destroy()
    budget = int(sorted(sizes)[-1] + sorted(sizes)[-2])      # two of the largest at most
    srv = sic.Server(hbm_budget=budget, max_active=8, chunk_steps=8)
    for p in probs:
        srv.sic_server_submit_horizontal(p)
    peak_active = 0
    while srv.sic_server_tick() > 0:
        st = srv.sic_server_stats()
        assert st["bytes_in_use"] <= budget
        peak_active = max(peak_active, st["active"])
    res = srv.sic_server_results()
    st = srv.sic_server_stats()
    srv.sic_server_destroy()
    assert len(res) == len(probs) and all(r["status"] == 0 for r in res)
    assert st["bytes_peak"] <= budget
    assert peak_active >= 2


def test_oversize_request_is_refused(sic):
    p = _mix(1, seed=5)[0]
    srv = sic.Server(hbm_budget=4096, max_active=2, chunk_steps=8)
    srv.sic_server_submit_horizontal(p)
    while srv.sic_server_tick() > 0:
        pass
    res = srv.sic_server_results()
    srv.sic_server_destroy()
    assert len(res) == 1 and res[0]["status"] == sic.SIC_EBUSY


def test_midrun_arrivals_join_the_batch(sic):
    probs = _mix(6, seed=21)
    for p in probs:
        p.n_steps = 64
    srv = sic.Server(hbm_budget=8 << 30, max_active=8, chunk_steps=8)
    first = [srv.sic_server_submit_horizontal(p) for p in probs[:3]]
    srv.sic_server_tick()
    assert srv.sic_server_stats()["active"] == 3
    later = [srv.sic_server_submit_horizontal(p) for p in probs[3:]]
    srv.sic_server_tick()
    st = srv.sic_server_stats()
    assert st["active"] == 6          # the newcomers run alongside the first three
    while srv.sic_server_tick() > 0:
        pass
    res = {r["id"]: r for r in srv.sic_server_results()}
    srv.sic_server_destroy()
    assert all(res[i]["status"] == 0 for i in first + later)
    # the first three finish before the later ones, which started 8 steps behind
    assert max(res[i]["t_done"] for i in first) <= min(res[i]["t_done"] for i in later)
    assert min(res[i]["t_admit"] for i in later) < max(res[i]["t_done"] for i in first)


def test_trace_replay_latencies(sic):
    from paper_1506_07207_gb300 import serving
    reqs = inputs.serving_mix(n_requests=12, seed=9, rate=200.0, max_sheets_exp=7, max_tracers_exp=12,
                              max_nx_exp=10, min_steps=20, max_steps=80)
    probs = [r.problem() for r in reqs]
    arr = [r.arrival for r in reqs]
    out = serving.run_trace(probs, arr, plain=False, max_active=16, chunk_steps=16)
    assert np.all(out["latency_s"] > 0)
    assert out["segment_updates"] == sum(p.n_segments * p.n_steps for p in probs)
    assert out["p99_ms"] >= out["p50_ms"] > 0


def test_refining_requests_equal_alone_and_plain(sic):
    """Requests whose sheets stretch past their refinement length (Sec. 2.6)
    hold at their own step, are refined by the server and go on; each ends
    with the same bits as the same request run alone with sic_run, batched or
    plain, and its segment-updates count the segments it had at every step."""
    probs = []
    for i, (v0, k) in enumerate([(1.5, 0.4), (1.2, 0.5), (2.0, 0.3)]):
        p = inputs.two_stream(v0, 0.05, k, nx=128, n_sheets=16, n_tracers=512, eps=0.05, t_end=25.0 + 2 * i)
        p.refine_length = 2.0 * p.L / p.nx
        probs.append(p)
    probs += _mix(3, seed=13)
    alone = []
    for p in probs:
        sim = sic.Sim.from_problem(p, history_len=1)
        try:
            added = sim.sic_run(p.n_steps)
            alone.append((_key(sim.sic_diagnostics()), sim.sic_get_state(), added))
        finally:
            sim.sic_destroy()
    assert all(a[2] > 0 for a in alone[:3])            # the stretched ones did refine
    for plain in (False, True):
        srv = sic.Server(hbm_budget=8 << 30, max_active=8, chunk_steps=16, plain=plain)
        ids = [srv.sic_server_submit_horizontal(p, keep=True) for p in probs]
        got = {}
        while srv.sic_server_tick() > 0:
            for r in srv.sic_server_results():
                got[r["id"]] = r
        for r in srv.sic_server_results():
            got[r["id"]] = r
        st = srv.sic_server_stats()
        srv.sic_server_destroy()
        for rid, p, (key, (x, v), added) in zip(ids, probs, alone):
            r = got[rid]
            assert r["status"] == 0 and r["steps"] == p.n_steps
            assert (r["field_energy"], r["kinetic_energy"], r["momentum"], r["charge_fixed"]) == key
            kept = sic.adopt_sim(r["sim"], p.nx, np.full(p.n_sheets, 1))
            try:
                kept._update_counts()
                xg, vg = kept.sic_get_state()
                np.testing.assert_array_equal(xg, x)
                np.testing.assert_array_equal(vg, v)
            finally:
                kept.sic_destroy()
            if added == 0:
                assert r["segment_updates"] == p.n_segments * p.n_steps
            else:
                assert r["segment_updates"] > p.n_segments * p.n_steps
        assert st["bytes_in_use"] == 0


def test_request_at_its_tracer_limit_ends_with_its_steps(sic):
    """A served request whose refinement would pass its tracer limit ends
    there with SIC_ELIMIT and the steps it took; the others are unaffected."""
    p = inputs.two_stream(1.5, 0.05, 0.4, nx=128, n_sheets=16, n_tracers=512, eps=0.05, t_end=30.0)
    p.refine_length = 2.0 * p.L / p.nx
    p.max_tracers = p.n_tracers + 40
    others = _mix(3, seed=17)
    srv = sic.Server(hbm_budget=8 << 30, max_active=8, chunk_steps=16)
    rid = srv.sic_server_submit_horizontal(p)
    oids = [srv.sic_server_submit_horizontal(q) for q in others]
    while srv.sic_server_tick() > 0:
        pass
    res = {r["id"]: r for r in srv.sic_server_results()}
    srv.sic_server_destroy()
    assert res[rid]["status"] == sic.SIC_ELIMIT and 0 < res[rid]["steps"] < p.n_steps
    assert all(res[i]["status"] == 0 and res[i]["steps"] == q.n_steps for i, q in zip(oids, others))


def test_zero_step_and_kept_requests(sic):
    """In long chunks every request ends at its own length, a request of zero
    steps is done as it stands, and a kept simulation steps on normally once
    handed over."""
    probs = _mix(6, seed=23)
    srv = sic.Server(hbm_budget=8 << 30, max_active=6, chunk_steps=64)
    ids = [srv.sic_server_submit_horizontal(p, keep=(i == 0)) for i, p in enumerate(probs)]
    zero = srv.sic_server_submit_horizontal(probs[1], n_steps=0)
    got = {}
    while srv.sic_server_tick() > 0:
        for r in srv.sic_server_results():
            got[r["id"]] = r
    for r in srv.sic_server_results():
        got[r["id"]] = r
    srv.sic_server_destroy()
    assert got[zero]["status"] == 0 and got[zero]["steps"] == 0 and got[zero]["segment_updates"] == 0
    for rid, p in zip(ids, probs):
        r = got[rid]
        assert r["status"] == 0 and r["steps"] == p.n_steps
        assert (r["field_energy"], r["kinetic_energy"], r["momentum"], r["charge_fixed"]) == _key(_alone(sic, p))
    kept = sic.adopt_sim(got[ids[0]]["sim"], probs[0].nx, probs[0].counts)
    ref = sic.Sim.from_problem(probs[0], history_len=1)
    try:
        kept.sic_step(5)
        ref.sic_step(probs[0].n_steps + 5)
        # (both hold at the same step if a particle passes the refinement length)
        assert kept.sic_diagnostics()["step"] == ref.sic_diagnostics()["step"] > probs[0].n_steps
        assert _key(kept.sic_diagnostics()) == _key(ref.sic_diagnostics())
    finally:
        kept.sic_destroy()
        ref.sic_destroy()
