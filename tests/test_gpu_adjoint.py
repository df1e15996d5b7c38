"""The adjoint kernels against the FP64 oracle's central finite differences
(h = 1e-6) and against M^{-1} w (d qdd / d tau = M^{-1}, symmetric)."""
import numpy as np
import pytest

import oracle
from paper_1609_06779_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
H = 1e-6


def _decompose(J):
    """mass, COM and rotational inertia about the COM from a rigid-body J."""
    m = J[5, 5]
    C = J[:3, 3:] / m
    c = np.array([C[2, 1], C[0, 2], C[1, 0]])
    Ic = J[:3, :3] + m * (C @ C)
    return m, c, Ic


def _with_mass(model, link, dm):
    J = model.inertias.copy()
    m, c, Ic = _decompose(J[link].reshape(6, 6))
    J[link] = synth.rigid_body_inertia(np.array(m + dm), c, Ic).reshape(36)
    return synth.ChainModel(model.axes, model.frames, J, model.offsets, model.gravity)


def _oracle_vjp(model, st, w):
    """Central-difference Jacobians of the oracle's qdd, contracted with w."""
    f = lambda m, q, qd, tau: oracle.fd(m, q, qd, tau)
    L = model.n_links_total
    gq, gqd, gm = np.zeros(L), np.zeros(L), np.zeros(L)
    for j in range(L):
        e = np.zeros(L); e[j] = H
        gq[j] = w @ (f(model, st.q + e, st.qdot, st.tau) - f(model, st.q - e, st.qdot, st.tau)) / (2 * H)
        gqd[j] = w @ (f(model, st.q, st.qdot + e, st.tau) - f(model, st.q, st.qdot - e, st.tau)) / (2 * H)
        gm[j] = w @ (f(_with_mass(model, j, H), st.q, st.qdot, st.tau)
                     - f(_with_mass(model, j, -H), st.q, st.qdot, st.tau)) / (2 * H)
    return gq, gqd, gm


@pytest.mark.parametrize("algo", ["abia", "jsiia", "cfa", "cfa_cr", "cfa_hybrid"])
@pytest.mark.parametrize("team", [1, 4, 8])
def test_adjoint_matches_oracle_finite_differences(algo, team):
    if algo == "abia" and team == 4:
        pytest.skip("ABIA teams are 1, 8, 16, 32")
    from paper_1609_06779_gb300 import fd
    model = synth.random_chains([1, 3, 7, 12], seed=41)
    st = synth.random_states(model.n_links_total, seed=42)
    w = np.random.default_rng(43).standard_normal(model.n_links_total)
    gq, gqd, gm = _oracle_vjp(model, st, w)
    cs = fd.ChainSet(model)
    b = fd.Batch(cs)
    t = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")
    qb, qdb, tb, mb = fd.adjoint(b, t(st.q), t(st.qdot), t(st.tau), t(w), algo=algo, team=team)
    torch.cuda.synchronize()
    for name, got, ref in (("q", qb, gq), ("qdot", qdb, gqd), ("mass", mb, gm)):
        got = got.cpu().numpy()
        for k in range(model.n_chains):
            a, c = model.offsets[k], model.offsets[k + 1]
            scale = max(np.abs(ref[a:c]).max(), 1e-8)
            assert np.abs(got[a:c] - ref[a:c]).max() / scale < 1e-6, (name, k)
    # tau_bar = M^{-1} w, chain by chain
    tb = tb.cpu().numpy()
    for k in range(model.n_chains):
        a, c = model.offsets[k], model.offsets[k + 1]
        M = oracle.mass_matrix(model.chain(k), st.q[a:c])
        np.testing.assert_allclose(tb[a:c], np.linalg.solve(M, w[a:c]), rtol=1e-9, atol=1e-11)


def test_adjoint_reuses_forward_result_and_algorithms_agree():
    from paper_1609_06779_gb300 import fd
    model = synth.random_chains([32] * 64 + [5, 17], seed=51)
    st = synth.random_states(model.n_links_total, seed=52)
    w = np.random.default_rng(53).standard_normal(model.n_links_total)
    cs = fd.ChainSet(model)
    b = fd.Batch(cs)
    t = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")
    q, qd, tau, wt = t(st.q), t(st.qdot), t(st.tau), t(w)
    ref = fd.adjoint(b, q, qd, tau, wt, algo="cfa", team=32)
    qdd = fd.solve(b, q, qd, tau, algo="jsiia")
    for algo, team in (("abia", 1), ("abia", 16), ("jsiia", 8), ("cfa", 1)):
        got = fd.adjoint(b, q, qd, tau, wt, qdd=qdd, algo=algo, team=team)
        for x, y in zip(got, ref):
            x, y = x.cpu().numpy(), y.cpu().numpy()
            assert np.abs(x - y).max() <= 1e-8 * max(np.abs(y).max(), 1.0), algo


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_shared_elimination_equals_separate_solves(prec):
    """Without a given qdd the adjoint solves FD and lambda = M^-1 w in one
    elimination (two right-hand sides); the results equal a separate FD solve and
    the adjoint given that qdd (one linear solve) bitwise, for every algorithm
    and for scan and component-lane teams."""
    from paper_1609_06779_gb300 import fd
    model = synth.random_chains([1, 5, 20, 33, 70, 32, 32], seed=61)
    st = synth.random_states(model.n_links_total, seed=62)
    w = np.random.default_rng(63).standard_normal(model.n_links_total)
    cs = fd.ChainSet(model)
    b = fd.Batch(cs)
    dt = torch.float64 if prec == "fp64" else torch.float32
    t = lambda a: torch.tensor(a, dtype=dt, device="cuda")
    q, qd, tau, wt = t(st.q), t(st.qdot), t(st.tau), t(w)
    for algo, team in (("abia", 1), ("abia", 8), ("abia", 16), ("jsiia", 2), ("jsiia", 8),
                       ("cfa", 8), ("cfa", 64), ("cfa_cr", 4)):
        qdd = fd.solve(b, q, qd, tau, algo=algo, prec=prec, team=team)
        one = fd.adjoint(b, q, qd, tau, wt, algo=algo, prec=prec, team=team, masses=False)
        two = fd.adjoint(b, q, qd, tau, wt, qdd=qdd, algo=algo, prec=prec, team=team,
                         masses=False)
        for k, (x, y) in enumerate(zip(one, two)):
            if x is None:
                continue
            assert torch.equal(x, y), (algo, team, k)


def test_autograd_function_gradcheck_direction():
    """torch.autograd through forward_dynamics: directional derivative of
    <w, qdd> along a random unit direction equals Richardson-extrapolated central
    differences of the GPU solve."""
    from paper_1609_06779_gb300 import fd
    model = synth.random_chains([6, 9], seed=61)
    st = synth.random_states(model.n_links_total, seed=62)
    cs = fd.ChainSet(model)
    b = fd.Batch(cs)
    rng = np.random.default_rng(63)
    t = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")
    q, qd, tau = (t(x).requires_grad_(True) for x in (st.q, st.qdot, st.tau))
    w = t(rng.standard_normal(model.n_links_total))
    qdd = fd.forward_dynamics(b, q, qd, tau, algo="cfa")
    (qdd * w).sum().backward()
    for idx, x in enumerate((q, qd, tau)):
        d = rng.standard_normal(model.n_links_total)
        d = t(d / np.linalg.norm(d))
        args = [q.detach(), qd.detach(), tau.detach()]

        def central(step):
            up = list(args); up[idx] = args[idx] + step * d
            dn = list(args); dn[idx] = args[idx] - step * d
            return float(((fd.solve(b, *up) - fd.solve(b, *dn)) * w).sum()) / (2 * step)

        with torch.no_grad():
            # Richardson at h = 1e-4 (O(h^4)); at 1e-6 the rounding of the two FP64
            # solves, divided by 2h, would be about 1e-5 of the result
            num = (4 * central(5e-5) - central(1e-4)) / 3
        ana = float((x.grad * d).sum())
        assert abs(ana - num) <= 1e-6 * max(abs(num), 1.0), (idx, ana, num)
