"""Kinematic trees (fd_create_tree): ABIA, JSIIA and inverse dynamics over a
parent array on the GPU, one thread per tree, called through the C ABI and
checked against the oracle's dense definitions over the same parent array
(oracle.fd_tree, oracle.rnea_tree)."""
import numpy as np
import pytest

import oracle
import oracle.dense as dense
from paper_1609_06779_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

EPS64 = float(np.finfo(np.float64).eps)
EPS32 = float(np.finfo(np.float32).eps)
SIZES = [1, 2, 3, 5, 8, 13, 31, 32, 33, 64, 100]


def _rel_err(got, ref, offsets):
    errs = []
    for p in range(len(offsets) - 1):
        a, b = offsets[p], offsets[p + 1]
        if b == a:
            continue
        scale = max(np.abs(ref[a:b]).max(), 1e-300)
        errs.append(np.abs(got[a:b] - ref[a:b]).max() / scale)
    return np.array(errs)


def _cond(model, q):
    out = []
    for p in range(model.n_chains):
        a, z = model.offsets[p], model.offsets[p + 1]
        out.append(np.linalg.cond(dense.mass_matrix(model.chain(p), q[a:z])) if z > a else 1.0)
    return np.array(out)


def _solve(model, st, algo, prec, team=0):
    from paper_1609_06779_gb300 import fd
    cs = fd.ChainSet(model)
    b = fd.Batch(cs)
    dt = torch.float64 if prec == "fp64" else torch.float32
    q, qd, tau = (torch.tensor(x, dtype=dt, device="cuda") for x in (st.q, st.qdot, st.tau))
    status = torch.full((b.n_problems,), -1, dtype=torch.int32, device="cuda")
    out = fd.solve(b, q, qd, tau, algo=algo, prec=prec, team=team, status=status)
    torch.cuda.synchronize()
    return out.double().cpu().numpy(), status.cpu().numpy()


@pytest.mark.parametrize("algo", ["abia", "jsiia"])
def test_tree_fd_fp64_parity(algo):
    model = synth.random_trees(SIZES * 2, seed=41)
    st = synth.random_states(model.n_links_total, seed=42)
    ref = oracle.fd_tree(model, st.q, st.qdot, st.tau)
    got, status = _solve(model, st, algo, "fp64")
    assert (status == 0).all()
    err = _rel_err(got, ref, model.offsets)
    # a backward-stable solve loses about cond(M) eps64
    tol = np.maximum(1e-10, 10 * _cond(model, st.q) * EPS64)
    assert (err <= tol).all(), (algo, err.max(), (err / tol).max())


def test_tree_inverse_dynamics_fp64_parity():
    from paper_1609_06779_gb300 import fd
    model = synth.random_trees(SIZES, seed=43)
    st = synth.random_states(model.n_links_total, seed=44)
    qdd = np.random.default_rng(45).standard_normal(model.n_links_total)
    ref = oracle.rnea_tree(model, st.q, st.qdot, qdd)
    b = fd.Batch(fd.ChainSet(model))
    t = lambda x: torch.tensor(x, dtype=torch.float64, device="cuda")
    tau = fd.inverse_dynamics(b, t(st.q), t(st.qdot), t(qdd))
    torch.cuda.synchronize()
    err = _rel_err(tau.cpu().numpy(), ref, model.offsets)
    assert err.max() < 1e-12, err.max()


def test_tree_with_chain_parents_matches_the_chain_path():
    """parents = i - 1 is the serial chain: the tree kernels agree with the chain
    kernels (other code, same model) to FP64 rounding."""
    chains = synth.random_chains(SIZES, seed=46)
    tree = synth.random_chains(SIZES, seed=46)
    tree.parents = np.concatenate([np.arange(n) - 1 for n in tree.lengths()]).astype(np.int32)
    st = synth.random_states(chains.n_links_total, seed=47)
    for algo in ("abia", "jsiia"):
        a, sa = _solve(chains, st, algo, "fp64", team=1)
        b, sb = _solve(tree, st, algo, "fp64")
        assert (sa == 0).all() and (sb == 0).all()
        err = _rel_err(b, a, chains.offsets)
        assert err.max() < 1e-10, (algo, err.max())


@pytest.mark.parametrize("algo", ["abia", "jsiia"])
def test_tree_fd_fp32_bars(algo):
    model = synth.random_trees([1, 2, 4, 7, 8, 13] * 6, seed=48)
    st = synth.random_states(model.n_links_total, seed=49)
    ref = oracle.fd_tree(model, st.q, st.qdot, st.tau)
    cond = _cond(model, st.q)
    good = cond * EPS32 <= 1e-4
    assert good.mean() > 0.8
    got, status = _solve(model, st, algo, "fp32")
    assert (status == 0).all()
    err = _rel_err(got, ref, model.offsets)
    assert err[good].max() < 1e-4, (algo, err[good].max())
    assert (err <= np.maximum(1e-4, 4 * cond * EPS32)).all()


def test_tree_unsupported_options():
    from paper_1609_06779_gb300 import fd
    model = synth.random_trees([5, 6], seed=50)
    st = synth.random_states(model.n_links_total, seed=51)
    b = fd.Batch(fd.ChainSet(model))
    t = lambda x, dt=torch.float64: torch.tensor(x, dtype=dt, device="cuda")
    q, qd, tau = t(st.q), t(st.qdot), t(st.tau)
    for algo in ("cfa", "cfa_cr", "cfa_hybrid", "abia_scan"):
        with pytest.raises(fd.FDError, match="kinematic trees"):
            fd.solve(b, q, qd, tau, algo=algo, ws=fd.workspace(b, "cfa"))
    with pytest.raises(fd.FDError, match="one thread per tree"):
        fd.solve(b, q, qd, tau, algo="abia", team=8)
    f = lambda x: t(x, torch.float32)
    with pytest.raises(fd.FDError, match="FP64 or FP32"):
        fd.solve(b, f(st.q), f(st.qdot), f(st.tau), algo="jsiia", prec="mixed")
    with pytest.raises(fd.FDError, match="serial chains only"):
        fd.solve_cfa_projected(b, q, qd, tau, projection="block_jacobi")
    with pytest.raises(fd.FDError):
        fd.adjoint(b, q, qd, tau, torch.ones_like(q), algo="abia")
    assert fd.autotune(b, q, qd, tau, algo="abia") == 1


def _looped(sizes, seed, per_tree=1):
    from paper_1609_06779_gb300 import fd
    model = synth.random_trees(sizes, seed=seed)
    loops = synth.random_loops(model, per_tree=per_tree, seed=seed + 1)
    st = synth.random_states(model.n_links_total, seed=seed + 2)
    cs = fd.ChainSet(model)
    cs.add_loops(loops)
    return fd, model, loops, st, cs


def test_looped_trees_jsiia_fp64_parity():
    """Trees closed by revolute loop joints (fd_tree_add_loops): the GPU's
    constrained accelerations against the oracle's dense KKT solve, and the
    constraints G qdd + gamma = 0 (the oracle's G, gamma) on the GPU result."""
    for sizes, seed, per_tree in (([12, 16, 24, 32, 40] * 3, 61, 1), ([32, 40, 48] * 3, 67, 2)):
        _check_looped(sizes, seed, per_tree)


def _check_looped(sizes, seed, per_tree):
    fd, model, loops, st, cs = _looped(sizes, seed=seed, per_tree=per_tree)
    b = fd.Batch(cs)
    t = lambda x: torch.tensor(x, dtype=torch.float64, device="cuda")
    status = torch.full((b.n_problems,), -1, dtype=torch.int32, device="cuda")
    got = fd.solve(b, t(st.q), t(st.qdot), t(st.tau), algo="jsiia", status=status)
    torch.cuda.synchronize()
    assert (status.cpu().numpy() == 0).all()
    got = got.cpu().numpy()
    ref = oracle.fd_looped(model, st.q, st.qdot, st.tau, loops)
    for p in range(model.n_chains):
        a, z = model.offsets[p], model.offsets[p + 1]
        sel = np.nonzero(loops["tree"] == p)[0]
        lp = {k: np.asarray(loops[k])[sel] for k in ("a", "b", "frame_a", "frame_b")}
        one = model.chain(p)
        M = dense.mass_matrix(one, st.q[a:z])
        G, gamma = dense.loop_constraints(one, st.q[a:z], st.qdot[a:z], lp)
        kkt = np.block([[M, G.T], [G, np.zeros((G.shape[0], G.shape[0]))]])
        tol = max(1e-10, 10 * np.linalg.cond(kkt) * EPS64)
        err = np.abs(got[a:z] - ref[a:z]).max() / np.abs(ref[a:z]).max()
        assert err <= tol, (p, err, tol)
        res = G @ got[a:z] + gamma
        assert np.abs(res).max() <= tol * max(np.abs(gamma).max(), np.abs(G).max() * np.abs(ref[a:z]).max())


def test_looped_set_trees_without_loops_and_options():
    """In a set with loops, a tree without one solves as an open tree; the other
    algorithms and precisions are refused, and loops are added once."""
    from paper_1609_06779_gb300 import fd
    sizes = [20, 9, 20]
    model = synth.random_trees(sizes, seed=63)
    loops = synth.random_loops(model, per_tree=1, seed=64)
    keep = loops["tree"] != 1
    loops = {k: np.asarray(v)[keep] for k, v in loops.items()}
    st = synth.random_states(model.n_links_total, seed=65)
    cs = fd.ChainSet(model)
    cs.add_loops(loops)
    b = fd.Batch(cs)
    t = lambda x, dt=torch.float64: torch.tensor(x, dtype=dt, device="cuda")
    q, qd, tau = t(st.q), t(st.qdot), t(st.tau)
    got = fd.solve(b, q, qd, tau, algo="jsiia").cpu().numpy()
    a, z = model.offsets[1], model.offsets[2]
    ref = oracle.fd_tree(model, st.q, st.qdot, st.tau)
    assert np.abs(got[a:z] - ref[a:z]).max() <= 1e-10 * np.abs(ref[a:z]).max()
    with pytest.raises(fd.FDError, match="loops run JSIIA"):
        fd.solve(b, q, qd, tau, algo="abia")
    f = lambda x: t(x, torch.float32)
    with pytest.raises(fd.FDError, match="loops run JSIIA"):
        fd.solve(b, f(st.q), f(st.qdot), f(st.tau), algo="jsiia", prec="fp32")
    with pytest.raises(fd.FDError, match="loops run JSIIA"):
        fd.inverse_dynamics(b, q, qd, tau)
    with pytest.raises(fd.FDError, match="already"):
        cs.add_loops(loops)
    chains = fd.ChainSet(synth.random_chains([20], seed=66))
    with pytest.raises(fd.FDError, match="not a set of kinematic trees"):
        chains.add_loops(loops)
    bad = dict(loops, b=np.full_like(loops["b"], 99))
    with pytest.raises(fd.FDError, match="links"):
        fd.ChainSet(model).add_loops(bad)


def test_tree_edge_cases_empty_and_single_link():
    """A set with an empty tree, a one-link tree and a link on the base beside a
    branch solves (status 0 for every problem, the empty tree untouched), and
    an empty batch is a no-op for the tree and projected solves."""
    from paper_1609_06779_gb300 import fd
    m = synth.random_trees([0, 1, 6, 0, 3], seed=71)
    m.parents[1 + 2] = -1  # a second link on the base in the 6-link tree
    st = synth.random_states(m.n_links_total, seed=72)
    ref = oracle.fd_tree(m, st.q, st.qdot, st.tau)
    for algo in ("abia", "jsiia"):
        got, status = _solve(m, st, algo, "fp64")
        assert (status == 0).all()
        err = _rel_err(got, ref, m.offsets)
        assert err.max() < 1e-12, (algo, err.max())
    empty = synth.random_trees([0, 0], seed=73)
    b = fd.Batch(fd.ChainSet(empty))
    z = torch.zeros(0, dtype=torch.float64, device="cuda")
    for algo in ("abia", "jsiia"):
        assert fd.solve(b, z, z, z, algo=algo).numel() == 0
    cb = fd.Batch(fd.ChainSet(synth.random_chains([0, 0], seed=74)))
    assert fd.solve_cfa_projected(cb, z, z, z, projection="block_jacobi").numel() == 0
