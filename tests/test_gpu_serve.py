"""The serving runtime: each request's result is the same alone and in a mix,
agrees with the batch API, admission under a small budget, the timeout path."""
import numpy as np
import pytest

import oracle
from paper_1609_06779_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _requests(rng, n_models=12, n_req=60):
    lengths = synth.log_uniform_lengths(n_models, 6, 64, seed=int(rng.integers(1 << 30)))
    models = [synth.random_chains([int(n)], seed=100 + k) for k, n in enumerate(lengths)]
    reqs = []
    for r in range(n_req):
        k = int(rng.integers(n_models))
        n = int(lengths[k])
        st = synth.random_states(n, seed=1000 + r)
        algo = ("abia", "cfa")[r % 2]
        if r % 3 == 0:
            steps = int(rng.integers(1, 8))
            taus = rng.standard_normal((steps, n)) * 10
            reqs.append(dict(kind="rollout", model=k, q=st.q, qd=st.qdot, taus=taus, dt=1e-3,
                             algo=algo))
        else:
            reqs.append(dict(kind="grad", model=k, q=st.q, qd=st.qdot, tau=st.tau,
                             w=rng.standard_normal(n), algo=algo))
    return models, reqs


def _run(server, ids, reqs):
    tickets = []
    for r in reqs:
        if r["kind"] == "rollout":
            tickets.append(server.submit_rollout(ids[r["model"]], r["q"], r["qd"], r["taus"],
                                                 r["dt"], algo=r["algo"]))
        else:
            tickets.append(server.submit_grad(ids[r["model"]], r["q"], r["qd"], r["tau"], r["w"],
                                              algo=r["algo"]))
    return [server.wait(t, timeout_ms=60000) for t in tickets]


def test_each_result_is_the_same_alone_and_in_the_mix():
    from paper_1609_06779_gb300 import fd
    rng = np.random.default_rng(0)
    models, reqs = _requests(rng)
    srv = fd.Server(budget_bytes=256 << 20)
    ids = [srv.add_model(m) for m in models]
    mixed = _run(srv, ids, reqs)
    for r, res in zip(reqs[:20], mixed[:20]):
        alone = _run(srv, ids, [r])[0]
        assert res["status"] == 0 and alone["status"] == 0
        keys = ("q", "qdot", "qddot") if r["kind"] == "rollout" else (
            "qddot", "q_bar", "qdot_bar", "tau_bar")
        for k in keys:
            assert np.array_equal(res[k], alone[k]), (r["kind"], k)
    st = srv.stats()
    assert st["completed"] == len(reqs) + 20 and st["active"] == 0
    srv.close()


def test_every_team_class_alone_and_in_the_mix():
    """Chains of 6..256 links fall into every team class of the server (and onto
    every side stream); each result is bitwise the same alone and in the mix."""
    from paper_1609_06779_gb300 import fd
    rng = np.random.default_rng(3)
    lengths = [6, 20, 40, 60, 100, 128, 160, 256]
    models = [synth.random_chains([n], seed=300 + k) for k, n in enumerate(lengths)]
    reqs = []
    for r in range(24):
        k = r % len(lengths)
        n = lengths[k]
        st = synth.random_states(n, seed=3000 + r)
        algo = ("cfa", "abia")[(r // len(lengths)) % 2]
        if r % 3 == 2:
            reqs.append(dict(kind="rollout", model=k, q=st.q, qd=st.qdot,
                             taus=rng.standard_normal((3, n)) * 10, dt=1e-3, algo=algo))
        else:
            reqs.append(dict(kind="grad", model=k, q=st.q, qd=st.qdot, tau=st.tau,
                             w=rng.standard_normal(n), algo=algo))
    srv = fd.Server(budget_bytes=256 << 20)
    ids = [srv.add_model(m) for m in models]
    mixed = _run(srv, ids, reqs)
    for r, res in zip(reqs, mixed):
        alone = _run(srv, ids, [r])[0]
        assert res["status"] == 0 and alone["status"] == 0
        keys = ("q", "qdot", "qddot") if r["kind"] == "rollout" else (
            "qddot", "q_bar", "qdot_bar", "tau_bar")
        for k in keys:
            assert np.array_equal(res[k], alone[k]), (r["kind"], lengths[r["model"]], k)
    srv.close()


def test_per_size_baseline_computes_the_same_results():
    """FD_SERVE_PER_SIZE (one launch per distinct length, the static baseline)
    runs the same kernels with the same teams: results bitwise equal."""
    from paper_1609_06779_gb300 import fd
    rng = np.random.default_rng(5)
    models, reqs = _requests(rng, n_models=8, n_req=30)
    out = []
    for per_size in (False, True):
        srv = fd.Server(budget_bytes=256 << 20, per_size=per_size)
        ids = [srv.add_model(m) for m in models]
        out.append(_run(srv, ids, reqs))
        srv.close()
    for r, a, b in zip(reqs, out[0], out[1]):
        assert a["status"] == 0 and b["status"] == 0
        keys = ("q", "qdot", "qddot") if r["kind"] == "rollout" else (
            "qddot", "q_bar", "qdot_bar", "tau_bar")
        for k in keys:
            assert np.array_equal(a[k], b[k]), (r["kind"], k)


def test_served_results_agree_with_the_batch_api_and_oracle():
    from paper_1609_06779_gb300 import fd
    rng = np.random.default_rng(1)
    models, reqs = _requests(rng, n_models=6, n_req=24)
    srv = fd.Server(budget_bytes=128 << 20)
    ids = [srv.add_model(m) for m in models]
    out = _run(srv, ids, reqs)
    t = lambda a: torch.tensor(np.asarray(a), dtype=torch.float64, device="cuda")
    for r, res in zip(reqs, out):
        m = models[r["model"]]
        cs = fd.ChainSet(m)
        b = fd.Batch(cs)
        n = m.n_links_total  # the server's rule
        team = (16 if n <= 64 else 32) if r["algo"] == "abia" else (
            8 if n <= 32 else (32 if n <= 64 else (64 if n <= 128 else 128)))
        if r["kind"] == "grad":
            ref = oracle.fd(m, r["q"], r["qd"], r["tau"])
            assert np.abs(res["qddot"] - ref).max() <= 1e-10 * max(np.abs(ref).max(), 1.0)
            qb, qdb, tb, _ = fd.adjoint(b, t(r["q"]), t(r["qd"]), t(r["tau"]), t(r["w"]),
                                        algo=r["algo"], team=team, masses=False)
            for k, x in (("q_bar", qb), ("qdot_bar", qdb), ("tau_bar", tb)):
                x = x.cpu().numpy()
                assert np.abs(res[k] - x).max() <= 1e-12 * max(np.abs(x).max(), 1.0), k
        else:
            q, qd = r["q"].copy(), r["qd"].copy()
            for tau in r["taus"]:   # semi-implicit Euler with the oracle
                qdd = oracle.fd(m, q, qd, tau)
                qd = qd + r["dt"] * qdd
                q = q + r["dt"] * qd
            np.testing.assert_allclose(res["q"], q, rtol=1e-10, atol=1e-10)
            np.testing.assert_allclose(res["qdot"], qd, rtol=1e-9, atol=1e-9)
            assert res["steps_done"] == len(r["taus"])
    srv.close()


def test_rollouts_over_several_ticks_follow_the_euler_loop():
    """Rollouts longer than a tick's steps (shorter chains take several steps per
    tick, the longest one) end where a semi-implicit Euler loop over the oracle
    does, for every length class and both algorithms."""
    from paper_1609_06779_gb300 import fd
    rng = np.random.default_rng(9)
    lengths = [6, 18, 30, 50, 90]
    models = [synth.random_chains([n], seed=900 + k) for k, n in enumerate(lengths)]
    srv = fd.Server(budget_bytes=128 << 20)
    ids = [srv.add_model(m) for m in models]
    reqs = []
    for k, n in enumerate(lengths):
        for algo in ("abia", "cfa"):
            st = synth.random_states(n, seed=9000 + 10 * k + len(reqs))
            steps = 23 if algo == "abia" else 11
            reqs.append(dict(kind="rollout", model=k, q=st.q, qd=st.qdot,
                             taus=rng.standard_normal((steps, n)) * 10, dt=1e-3, algo=algo))
    out = _run(srv, ids, reqs)
    for r, res in zip(reqs, out):
        m = models[r["model"]]
        q, qd = r["q"].copy(), r["qd"].copy()
        for tau in r["taus"]:
            qdd = oracle.fd(m, q, qd, tau)
            qd = qd + r["dt"] * qdd
            q = q + r["dt"] * qd
        assert res["status"] == 0 and res["steps_done"] == len(r["taus"])
        np.testing.assert_allclose(res["q"], q, rtol=1e-10, atol=1e-10)
        np.testing.assert_allclose(res["qdot"], qd, rtol=1e-9, atol=1e-9)
        np.testing.assert_allclose(res["qddot"], qdd, rtol=1e-9, atol=1e-9)
    srv.close()


def test_admission_under_a_small_budget_and_timeouts():
    from paper_1609_06779_gb300 import fd
    srv = fd.Server(budget_bytes=16 << 20)       # a few thousand link slots
    slots = srv.stats()["link_slots"]
    m = synth.random_chains([200], seed=5)
    mid = srv.add_model(m)
    rng = np.random.default_rng(2)
    n_req = int(3 * slots / 200) + 1             # three times what fits at once
    tickets = []
    for k in range(n_req):
        st = synth.random_states(200, seed=k)
        taus = rng.standard_normal((20, 200)) * 10
        tickets.append(srv.submit_rollout(mid, st.q, st.qdot, taus, 1e-3))
    # a bounded wait on the last request ends with FD_ERR_TIMEOUT, not a hang
    with pytest.raises(fd.FDError) as ei:
        srv.wait(tickets[-1], timeout_ms=1)
    assert ei.value.status == 5
    res = [srv.wait(tk, timeout_ms=120000) for tk in tickets]
    assert all(r["status"] == 0 and r["steps_done"] == 20 for r in res)
    assert srv.stats()["link_slots_used"] == 0
    with pytest.raises(fd.FDError):              # unknown model id
        srv.remove_model(12345)
    srv.remove_model(mid)
    srv.close()


def test_invalid_requests_are_refused():
    from paper_1609_06779_gb300 import fd
    srv = fd.Server(budget_bytes=32 << 20)
    m = synth.random_chains([5], seed=1)
    mid = srv.add_model(m)
    z = np.zeros(5)
    with pytest.raises(fd.FDError) as ei:
        srv.submit_grad(mid + 7, z, z, z, z)
    assert ei.value.status == 1
    with pytest.raises(fd.FDError) as ei:
        srv.submit_grad(mid, z, z, z, z, algo="jsiia")
    assert ei.value.status == 8
    with pytest.raises(fd.FDError):
        srv.submit_rollout(mid, z, z, np.zeros((3, 5)), dt=0.0)
    srv.close()
