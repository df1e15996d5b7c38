"""One launch over a batch of several length classes (team 0): the grid is
split by class and each class runs its own team. Checked against the oracle,
bit for bit against the single-team launch of the same team per class, through
the adjoint, after per-class autotuning, and under CUDA-graph capture."""
import numpy as np
import pytest

import oracle
from paper_1609_06779_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

LENGTHS = [1, 2, 3, 5, 6, 7, 8, 9, 13, 17, 31, 32, 33, 47, 64, 65, 100, 129, 200, 0] * 3


def _rel_err(got, ref, offsets):
    errs = []
    for p in range(len(offsets) - 1):
        a, b = offsets[p], offsets[p + 1]
        if b > a:
            errs.append(np.abs(got[a:b] - ref[a:b]).max() / max(np.abs(ref[a:b]).max(), 1e-300))
    return np.array(errs)


def _setup(lengths, seed, dt=torch.float64):
    from paper_1609_06779_gb300 import fd
    model = synth.random_chains(lengths, seed=seed)
    st = synth.random_states(model.n_links_total, seed=seed + 1)
    cs = fd.ChainSet(model)
    b = fd.Batch(cs)
    t = lambda a: torch.tensor(a, dtype=dt, device="cuda")
    return fd, model, st, cs, b, t(st.q), t(st.qdot), t(st.tau)


@pytest.mark.parametrize("algo", ["abia", "jsiia", "cfa", "cfa_cr", "cfa_hybrid"])
def test_class_split_fp64_parity_and_bitwise(algo):
    fd, model, st, cs, b, q, qd, tau = _setup(LENGTHS, 41)
    classes = fd.batch_classes(b, algo)
    assert len(classes) >= 8 and sum(c["count"] for c in classes) == len(LENGTHS)
    status = torch.full((b.n_problems,), -1, dtype=torch.int32, device="cuda")
    out = fd.solve(b, q, qd, tau, algo=algo, team=0, status=status)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert (status.cpu().numpy() == 0).all()
    ref = oracle.fd(model, st.q, st.qdot, st.tau)
    aba = oracle.fd(model, st.q, st.qdot, st.tau, algo="aba")
    floor = _rel_err(aba, ref, model.offsets)
    if algo.startswith("cfa"):
        floor = np.maximum(floor, _rel_err(oracle.fd(model, st.q, st.qdot, st.tau, algo="cfa"),
                                           ref, model.offsets))
    err = _rel_err(got, ref, model.offsets)
    assert (err <= np.maximum(1e-10, 10 * floor)).all(), err.max()
    # every class's problems equal, bit for bit, a single-team launch at that team
    lens = np.diff(model.offsets)
    for c in classes:
        single = fd.solve(b, q, qd, tau, algo=algo, team=c["team"]).cpu().numpy()
        for p in np.nonzero((lens >= c["min_len"]) & (lens <= c["max_len"]))[0]:
            a_, z_ = model.offsets[p], model.offsets[p + 1]
            assert np.array_equal(got[a_:z_], single[a_:z_]), (algo, c, p)


@pytest.mark.parametrize("prec", ["fp32", "mixed"])
def test_class_split_float_paths(prec):
    fd, model, st, cs, b, q, qd, tau = _setup(LENGTHS, 43, torch.float32)
    ref = oracle.fd(model, st.q, st.qdot, st.tau)
    lens = np.diff(model.offsets)
    for algo in ("abia", "jsiia", "cfa", "cfa_cr", "cfa_hybrid"):
        got = fd.solve(b, q, qd, tau, algo=algo, prec=prec, team=0).double().cpu().numpy()
        err = _rel_err(got, ref, model.offsets)
        short = lens[lens > 0] <= 8
        assert err[short].max() < 1e-4, (algo, prec, err[short].max())
        assert np.isfinite(got).all()


def test_class_split_autotune_and_cache(tmp_path):
    fd, model, st, cs, b, q, qd, tau = _setup(LENGTHS * 20, 45)
    ref = oracle.fd(model, st.q, st.qdot, st.tau, n_threads=8)
    fd.autotune_cache_clear()
    for algo in ("abia", "cfa"):
        assert fd.autotune(b, q, qd, tau, algo=algo) == 0   # per class
        classes = fd.batch_classes(b, algo)
        for c in classes:
            assert c["team"] in ((1, 8, 16, 32) if algo == "abia" else (1, 2, 4, 8, 16, 32, 64, 128))
        got = fd.solve(b, q, qd, tau, algo=algo).cpu().numpy()
        assert _rel_err(got, ref, model.offsets).max() < 1e-9, algo
    path = tmp_path / "tune.json"
    fd.autotune_cache_save(str(path))
    fd.autotune_cache_clear()
    assert fd.autotune_cache_load(str(path)) >= 2
    # a new plan of the same batch takes its teams from the cache without timing
    b2 = fd.Batch(cs)
    assert fd.autotune(b2, q, qd, tau, algo="cfa") == 0
    assert [c["team"] for c in fd.batch_classes(b2, "cfa")] == \
        [c["team"] for c in fd.batch_classes(b, "cfa")]


def test_class_split_adjoint_matches_single_team():
    # chains of up to 64 links: well enough conditioned that two FP64 schedules
    # agree to 1e-9 (longer ones are checked by the uneven-batch adjoint test
    # against central differences, which also runs the class split)
    fd, model, st, cs, b, q, qd, tau = _setup([1, 2, 3, 5, 7, 8, 13, 17, 31, 33, 47, 64] * 3, 47)
    assert len(fd.batch_classes(b, "cfa")) > 1
    w = torch.randn_like(q)
    for algo in ("cfa", "abia"):
        split = fd.adjoint(b, q, qd, tau, w, algo=algo, team=0)
        one = fd.adjoint(b, q, qd, tau, w, algo=algo, team=8)
        # q_bar, qdot_bar, mass_bar: the adjoint's bar against the oracle's central
        # differences (1e-6; two FP64 schedules measured 2e-8 apart at 64 links);
        # tau_bar = M^-1 w is a plain FP64 solve
        for x, y, tol in zip(split, one, (1e-6, 1e-6, 1e-9, 1e-6)):
            xa, ya = x.cpu().numpy(), y.cpu().numpy()
            assert _rel_err(xa, ya, model.offsets).max() < tol, algo


def test_class_split_graph_capture():
    fd, model, st, cs, b, q, qd, tau = _setup(LENGTHS, 49)
    ws = fd.workspace(b, "cfa", "fp64", 0, q.device)
    out = torch.empty_like(q)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        fd.solve(b, q, qd, tau, algo="cfa", out=out, ws=ws)
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        fd.solve(b, q, qd, tau, algo="cfa", out=out, ws=ws)
    st2 = synth.random_states(model.n_links_total, seed=99)
    q.copy_(torch.tensor(st2.q, device="cuda"))
    g.replay()
    torch.cuda.synchronize()
    eager = fd.solve(b, q, qd, tau, algo="cfa", ws=ws)
    assert torch.equal(out, eager)
