"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

FP64 bar: max_i |qdd_i - qdd_i^ref| / max(||qdd^ref||_inf, 1e-300) per problem
<= 1e-10 (raised only by the oracle's own disagreement floor between its two
independent routes, Cholesky and ABA, times 10, where the chain is ill
conditioned). FP32 / mixed bar: 1e-4 on well-conditioned (short) chains."""
import numpy as np
import pytest

import oracle
from paper_1609_06779_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _fd():
    from paper_1609_06779_gb300 import fd
    return fd


def _rel_err(got, ref, offsets):
    errs = []
    for p in range(len(offsets) - 1):
        a, b = offsets[p], offsets[p + 1]
        if b == a:
            continue
        scale = max(np.abs(ref[a:b]).max(), 1e-300)
        errs.append(np.abs(got[a:b] - ref[a:b]).max() / scale)
    return np.array(errs)


def _floor(model, st, offsets, problems=None):
    """The oracle's own two-route disagreement per problem (Cholesky vs ABA)."""
    ref = oracle.fd(model, st.q, st.qdot, st.tau, algo="cholesky", problems=problems)
    aba = oracle.fd(model, st.q, st.qdot, st.tau, algo="aba", problems=problems)
    return ref, aba


def _run(model, st, algo, prec, team, chain_index=None):
    fd = _fd()
    cs = fd.ChainSet(model)
    b = fd.Batch(cs, chain_index)
    dt = torch.float64 if prec == "fp64" else torch.float32
    q = torch.tensor(st.q, dtype=dt, device="cuda")
    qd = torch.tensor(st.qdot, dtype=dt, device="cuda")
    tau = torch.tensor(st.tau, dtype=dt, device="cuda")
    status = torch.full((max(b.n_problems, 1),), -1, dtype=torch.int32, device="cuda")
    out = fd.solve(b, q, qd, tau, algo=algo, prec=prec, team=team, status=status)
    torch.cuda.synchronize()
    return out.double().cpu().numpy(), status.cpu().numpy()[:b.n_problems]


RAGGED = [1, 2, 3, 5, 7, 8, 13, 31, 32, 33, 47, 64, 100]


@pytest.mark.parametrize("algo", ["abia", "jsiia", "cfa", "cfa_cr", "cfa_hybrid"])
@pytest.mark.parametrize("team", [1, 2, 4, 8, 16, 32, 64, 128, 256])
def test_fd_fp64_ragged_parity(algo, team):
    if algo == "abia" and team not in (1, 8, 16, 32):
        pytest.skip("ABIA teams are 1, 8, 16, 32")
    model = synth.random_chains(RAGGED * 2, seed=7)
    st = synth.random_states(model.n_links_total, seed=8)
    ref, aba = _floor(model, st, model.offsets)
    got, status = _run(model, st, algo, "fp64", team)
    assert (status == 0).all()
    err = _rel_err(got, ref, model.offsets)
    floor = _rel_err(aba, ref, model.offsets)
    if algo.startswith("cfa"):  # CFA eliminates through A: its own oracle route's floor
        floor = np.maximum(floor, _rel_err(oracle.fd(model, st.q, st.qdot, st.tau, algo="cfa"),
                                           ref, model.offsets))
    tol = np.maximum(1e-10, 10 * floor)
    assert (err <= tol).all(), f"max err {err.max():.3e} (tol {tol[np.argmax(err - tol)]:.3e})"


EPS32 = float(np.finfo(np.float32).eps)


def _cond_m(model, st, problems):
    """cond(M) of each problem's mass matrix at its q (oracle, 2-norm): a solve in
    single precision that is backward stable loses at most about cond(M) eps32."""
    out = []
    for p in problems:
        a, b = model.offsets[p], model.offsets[p + 1]
        out.append(np.linalg.cond(oracle.mass_matrix(model.chain(p), st.q[a:b])) if b > a else 1.0)
    return np.array(out)


def _check_float_bars(err, cond, what):
    """The single-precision bars: 1e-4 on well-conditioned problems
    (cond(M) eps32 <= 1e-4), and on every problem the forward-error bound of a
    backward-stable solve, max(1e-4, 4 cond(M) eps32)."""
    good = cond * EPS32 <= 1e-4
    if good.any():
        assert err[good].max() < 1e-4, (what, err[good].max())
    bound = np.maximum(1e-4, 4 * cond * EPS32)
    assert (err <= bound).all(), (what, (err / bound).max())


@pytest.mark.parametrize("prec", ["fp32", "mixed"])
@pytest.mark.parametrize("algo", ["abia", "jsiia", "cfa", "cfa_cr", "cfa_hybrid"])
def test_fd_fp32_parity_short_chains(prec, algo):
    model = synth.random_chains([1, 2, 4, 7, 7, 7, 8] * 8, seed=11)
    st = synth.random_states(model.n_links_total, seed=12)
    ref = oracle.fd(model, st.q, st.qdot, st.tau)
    cond = _cond_m(model, st, range(model.n_chains))
    assert (cond * EPS32 <= 1e-4).mean() > 0.9  # almost all of them well conditioned
    for team in ([1, 8, 32] if algo == "abia" else [1, 2, 8]):
        got, status = _run(model, st, algo, prec, team)
        assert (status == 0).all()
        err = _rel_err(got, ref, model.offsets)
        assert np.median(err) < 1e-5, (team, np.median(err))
        _check_float_bars(err, cond, (algo, prec, team))


@pytest.mark.parametrize("team", [1, 2, 4, 8, 16, 32, 64, 128, 256])
def test_inverse_dynamics_fp64_parity(team):
    fd = _fd()
    model = synth.random_chains(RAGGED, seed=3)
    st = synth.random_states(model.n_links_total, seed=4)
    qdd = np.random.default_rng(5).standard_normal(model.n_links_total)
    ref = oracle.rnea_batch(model, st.q, st.qdot, qdd)
    cs = fd.ChainSet(model)
    b = fd.Batch(cs)
    t = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")
    out = fd.inverse_dynamics(b, t(st.q), t(st.qdot), t(qdd), prec="fp64", team=team)
    got = out.cpu().numpy()
    err = _rel_err(got, ref, model.offsets)
    assert err.max() < 1e-12, err.max()


def test_shared_model_batch_cfg_small():
    """One 7-link chain, many states (the shared-model batch)."""
    model = synth.random_chains([7], seed=0)
    ci, so = synth.replicate_model(model, 1024)
    st = synth.random_states(7 * 1024, seed=1)
    ref = oracle.fd(model, st.q, st.qdot, st.tau, chain_index=ci, state_offsets=so,
                    n_threads=8)
    for algo in ("abia", "jsiia", "cfa"):
        got, status = _run(model, st, algo, "fp64", 0, chain_index=ci)
        assert (status == 0).all()
        assert _rel_err(got, ref, so).max() < 1e-10, algo


def test_nonfinite_input_flags_only_its_problem():
    """A NaN or infinite torque, or a NaN joint angle, makes that problem's status
    nonzero; the other problems of the same launch solve as usual."""
    model = synth.random_chains([7, 32, 5, 32, 9], seed=31)
    st = synth.random_states(model.n_links_total, seed=32)
    ref = oracle.fd(model, st.q, st.qdot, st.tau)
    off = model.offsets
    bad = synth.States(st.q.copy(), st.qdot.copy(), st.tau.copy())
    bad.tau[off[1] + 3] = np.nan
    bad.tau[off[2]] = np.inf
    bad.q[off[4] + 8] = np.nan
    clean = [0, 3]
    for algo in ("abia", "jsiia", "cfa", "cfa_cr", "cfa_hybrid"):
        for prec, team in (("fp64", 1), ("fp64", 2), ("fp64", 8), ("mixed", 8), ("fp32", 1)):
            if algo == "abia" and team == 2:
                continue
            got, status = _run(model, bad, algo, prec, team)
            assert list(status != 0) == [False, True, True, False, True], (algo, prec, team, status)
            err = _rel_err(got, ref, off)[clean]
            assert np.isfinite(err).all(), (algo, prec, team, err)
            if prec == "fp64":
                assert err.max() < 1e-10, (algo, prec, team, err)
            else:
                _check_float_bars(err, _cond_m(model, st, clean), (algo, prec, team))


def test_all_algorithms_and_teams_agree():
    model = synth.random_chains([32] * 64, seed=21)
    st = synth.random_states(model.n_links_total, seed=22)
    base, _ = _run(model, st, "cfa", "fp64", 32)
    for algo, team in (("cfa", 1), ("cfa", 4), ("jsiia", 1), ("jsiia", 32), ("abia", 1),
                       ("abia", 8), ("abia", 32), ("cfa_cr", 1), ("cfa_cr", 8), ("cfa_cr", 32),
                       ("cfa_hybrid", 1), ("cfa_hybrid", 8), ("cfa_hybrid", 32)):
        got, _ = _run(model, st, algo, "fp64", team)
        assert _rel_err(got, base, model.offsets).max() < 1e-10, (algo, team)


def test_edge_cases_empty_and_single_link():
    fd = _fd()
    # a chain with zero links between others, single-link chains
    model = synth.random_chains([1, 0, 3, 1], seed=2)
    st = synth.random_states(model.n_links_total, seed=3)
    ref = oracle.fd(model, st.q, st.qdot, st.tau)
    for algo in ("abia", "jsiia", "cfa", "cfa_cr"):
        got, status = _run(model, st, algo, "fp64", 0)
        np.testing.assert_allclose(got, ref, rtol=1e-11, atol=1e-11)
        assert (status == 0).all()
    # an empty batch is a no-op
    cs = fd.ChainSet(model)
    b = fd.Batch(cs, np.zeros(0, dtype=np.int32))
    assert b.n_problems == 0 and b.n_state_links == 0
    e = torch.empty(0, dtype=torch.float64, device="cuda")
    fd.solve(b, e, e, e, algo="cfa")


def test_repeat_is_bitwise_deterministic():
    model = synth.random_chains([32] * 256, seed=5)
    st = synth.random_states(model.n_links_total, seed=6)
    for algo in ("abia", "jsiia", "cfa"):
        a, _ = _run(model, st, algo, "fp64", 0)
        b, _ = _run(model, st, algo, "fp64", 0)
        assert np.array_equal(a, b), algo


def test_cuda_graph_replay_matches_eager():
    """fd_solve_batch enqueues only kernels on the caller's stream (no allocation,
    no synchronisation), so it can be captured in a CUDA graph; replays with new
    inputs copied into the captured buffers give the eager results bitwise."""
    fd = _fd()
    model = synth.random_chains([7] * 64 + [33, 100], seed=81)
    cs = fd.ChainSet(model)
    b = fd.Batch(cs)
    t = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")
    st0 = synth.random_states(model.n_links_total, seed=82)
    q, qd, tau = t(st0.q), t(st0.qdot), t(st0.tau)
    for algo, team in (("abia", 8), ("jsiia", 8), ("cfa", 8), ("cfa_cr", 4), ("cfa_hybrid", 8)):
        ws = fd.workspace(b, algo, "fp64", team, q.device)
        out = torch.empty_like(q)
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            fd.solve(b, q, qd, tau, algo=algo, team=team, out=out, ws=ws)
        torch.cuda.current_stream().wait_stream(s)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            fd.solve(b, q, qd, tau, algo=algo, team=team, out=out, ws=ws)
        for seed in (83, 84):
            st = synth.random_states(model.n_links_total, seed=seed)
            q.copy_(t(st.q)); qd.copy_(t(st.qdot)); tau.copy_(t(st.tau))
            g.replay()
            torch.cuda.synchronize()
            eager = fd.solve(b, q, qd, tau, algo=algo, team=team, ws=ws)
            assert torch.equal(out, eager), (algo, seed)


def test_bad_arguments_raise():
    fd = _fd()
    model = synth.random_chains([4, 4], seed=0)
    cs = fd.ChainSet(model)
    b = fd.Batch(cs)
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(fd.FDError):
        fd.solve(b, x.float(), x, x)                       # wrong dtype
    with pytest.raises(fd.FDError):
        fd.solve(b, x[:7], x[:7], x[:7])                   # wrong size
    with pytest.raises(fd.FDError):
        fd.solve(b, x, x, x, algo="abia", team=4)          # ABIA teams are 1, 8, 16, 32
    with pytest.raises(fd.FDError):
        fd.solve(b, x, x, x, team=3)                       # not a power of two
    ws = fd.workspace(b, "cfa")
    with pytest.raises(fd.FDError):
        fd.solve(b, x, x, x, ws=ws[: ws.numel() // 2])     # workspace too small
    with pytest.raises(fd.FDError):
        fd.Batch(cs, np.array([0, 2], dtype=np.int32))     # chain index out of range


@pytest.mark.parametrize("prec", ["fp64", "fp32", "mixed"])
def test_full_size_uniform_batch_sampled(prec):
    """65 536 chains x 32 links in the launch configuration the benchmark times;
    256 sampled problems against the oracle, properties on all of them."""
    model = synth.random_chains([32] * 65536, seed=0)
    st = synth.random_states(model.n_links_total, seed=1)
    sample = np.random.default_rng(2).choice(65536, 256, replace=False)
    ref = oracle.fd(model, st.q, st.qdot, st.tau, problems=sample)
    aba = oracle.fd(model, st.q, st.qdot, st.tau, algo="aba", problems=sample)
    off = model.offsets
    idx = np.concatenate([np.arange(off[p], off[p + 1]) for p in sample])
    so = np.arange(len(sample) + 1) * 32
    floor = _rel_err(aba[idx], ref[idx], so)
    cond = _cond_m(model, st, sample) if prec != "fp64" else None
    for algo in ("abia", "jsiia", "cfa"):
        got, status = _run(model, st, algo, prec, 0)
        assert (status == 0).all(), algo
        assert np.isfinite(got).all(), algo
        err = _rel_err(got[idx], ref[idx], so)
        if prec == "fp64":
            tol = np.maximum(1e-10, 10 * floor)
            assert (err <= tol).all(), (algo, err.max())
        else:
            # 32-link chains have cond(M) 3e3 .. 8e4: none is "well conditioned" in
            # single precision, so the bound of a backward-stable solve applies
            _check_float_bars(err, cond, (algo, prec))
            if prec == "mixed":  # only the inverse dynamics runs in FP32
                assert err.max() < 1e-4, (algo, err.max())


def test_autotune_records_a_team_and_matches():
    fd = _fd()
    # one length class (17..32 links): one team for the whole batch
    model = synth.random_chains([32] * 2048 + [17] * 100, seed=71)
    st = synth.random_states(model.n_links_total, seed=72)
    cs = fd.ChainSet(model)
    b = fd.Batch(cs)
    t = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")
    q, qd, tau = t(st.q), t(st.qdot), t(st.tau)
    ref = oracle.fd(model, st.q, st.qdot, st.tau, n_threads=8)
    for algo in ("abia", "jsiia", "cfa"):
        best = fd.autotune(b, q, qd, tau, algo=algo)
        assert best in (1, 2, 4, 8, 16, 32), (algo, best)
        if algo == "abia":
            assert best in (1, 8, 16, 32)
        # team 0 now uses the tuned size: same workspace size as asking for it
        assert b.workspace_size(algo, "fp64", 0) == b.workspace_size(algo, "fp64", best)
        got = fd.solve(b, q, qd, tau, algo=algo).cpu().numpy()
        assert _rel_err(got, ref, model.offsets).max() < 1e-10, algo
