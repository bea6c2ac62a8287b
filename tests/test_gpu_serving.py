"""Serving on the GPU: runs of different grid sizes and materials admitted into a shared request loop give
the same result as each run alone (bitwise: every run has its own buffers and stream and every
reduction is deterministic), admission respects the HBM budget, and a Poisson stream completes."""
import numpy as np
import pytest

import nm_inputs as inp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nmgb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2411_11725_gb300 as nmgb
    nmgb.load()
    return nmgb


def _stream(count, seed=3, duration_scale=0.01, rate_hz=1.0):
    out = []
    for i, (t, p) in enumerate(inp.serving_requests(count, seed, rate_hz=rate_hz, duration_scale=duration_scale)):
        kw = dict(n=p.n, dx=p.dx, m0=inp.serving_m0(p), t_end=p.extra["t_end"], Ms=p.Ms, A=p.A, Ku=p.Ku,
                  axis=p.axis, alpha=p.alpha, gamma=p.gamma, h=p.h_uniform, terms=p.terms, rtol=p.extra["rtol"],
                  atol=p.extra["atol"], dt0=p.extra["dt0"], tag=i)
        out.append((t, kw))
    return out


def _by_tag(results):
    return {r["tag"]: r for r in results}


def test_mixed_results_equal_alone(nmgb):
    from paper_2411_11725_gb300.serve import Server
    stream = _stream(10)
    alone = {}
    with Server(hbm_budget_bytes=8 << 30, max_active=1) as s:
        for _, kw in stream:
            s.submit(**kw)
            (r,) = s.drain(1)
            assert r["status"] == 0, r["message"]
            alone[r["tag"]] = r
    with Server(hbm_budget_bytes=8 << 30, max_active=6) as s:
        for _, kw in stream:
            s.submit(**kw)
        mixed = _by_tag(s.drain(len(stream)))
        st = s.stats()
    assert st["peak_active"] > 1 and st["completed"] == len(stream) and st["failed"] == 0
    assert max(r["n_active_at_admit"] for r in mixed.values()) > 1
    for tag, a in alone.items():
        b = mixed[tag]
        assert b["status"] == 0, b["message"]
        assert a["n_accepted"] == b["n_accepted"] and a["n_rejected"] == b["n_rejected"]
        assert a["t_final"] == b["t_final"]
        assert np.array_equal(a["m"], b["m"]), tag
        assert abs(a["t_final"] - stream[tag][1]["t_end"]) <= 1e-9 * stream[tag][1]["t_end"]
        assert np.allclose(np.linalg.norm(b["m"], axis=-1), 1.0, atol=1e-12)


def test_served_run_equals_mesh_run_until(nmgb):
    """The served integration is the single-mesh integration: same steps, same state."""
    from paper_2411_11725_gb300.serve import Server
    _, kw = _stream(4)[2]
    with Server(hbm_budget_bytes=8 << 30, max_active=2) as s:
        s.submit(**kw)
        (r,) = s.drain(1)
    me = nmgb.Mesh(kw["n"], kw["dx"], nmgb.F32)
    me.set_material(kw["Ms"], kw["A"], kw["Ku"], kw["axis"], kw["alpha"], kw["gamma"])
    me.set_zeeman(kw["h"])
    me.set_terms(kw["terms"])
    me.set_state(kw["m0"], 0.0, kw["dt0"])
    _, na, nr = me.run_until(kw["t_end"], nmgb.DP54, kw["rtol"], kw["atol"], kw["dt0"])
    m, t, _ = me.get_state()
    me.close()
    assert (na, nr) == (r["n_accepted"], r["n_rejected"])
    assert np.array_equal(m, r["m"])


def test_admission_by_footprint(nmgb):
    from paper_2411_11725_gb300.serve import Server
    stream = _stream(8, seed=4)
    fps = [nmgb.footprint_bytes(kw["n"]) for _, kw in stream]
    budget = max(fps) + min(fps) // 2
    with Server(hbm_budget_bytes=budget, max_active=8) as s:
        for _, kw in stream:
            s.submit(**kw)
        res = s.drain(len(stream))
        st = s.stats()
    assert all(r["status"] == 0 for r in res), [r["message"] for r in res]
    assert st["peak_bytes"] <= budget
    # a request larger than the whole budget is refused, the others still run
    big = dict(stream[0][1], n=(256, 256, 8), m0=inp.serving_m0(inp.Problem("x", (256, 256, 8), (3e-9,) * 3, 8e5,
                                                                            1e-11, extra=dict(m0_dir=(0, 0, 1),
                                                                                              m0_seed=1))),
               tag=100)
    with Server(hbm_budget_bytes=nmgb.footprint_bytes((256, 256, 8)) - 1, max_active=2) as s:
        s.submit(**big)
        s.submit(**stream[1][1])
        res = _by_tag(s.drain(2))
    assert res[100]["status"] == nmgb.ERR_OOM and "budget" in res[100]["message"]
    assert res[1]["status"] == 0


def test_poisson_replay_completes(nmgb):
    from paper_2411_11725_gb300.serve import Server, replay
    stream = _stream(16, seed=5, rate_hz=200.0)
    with Server(hbm_budget_bytes=4 << 30, max_active=8) as s:
        res = replay(s, [(t, kw) for t, kw in stream], timeout_s=300)
        st = s.stats()
    assert len(res) == len(stream) and all(r["status"] == 0 for r in res)
    lat = np.array([r["latency_s"] for r in res])
    assert np.all(lat > 0) and np.all(lat >= np.array([r["run_s"] for r in res]))
    assert st["busy_s"] > 0 and st["active_s"] >= st["busy_s"]
