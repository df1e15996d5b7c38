"""ABIA with the articulated-inertia recursion as a parallel scan (FD_ABIA_SCAN):
the Riccati step of the articulated inertia composed as Schur complements, the
bias-force and acceleration recursions as affine scans. FP64 parity with the
oracle on ragged and long chains, and the options it does not support."""
import numpy as np
import pytest

import oracle
from paper_1609_06779_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _rel_err(got, ref, offsets):
    errs = []
    for p in range(len(offsets) - 1):
        a, b = offsets[p], offsets[p + 1]
        if b > a:
            errs.append(np.abs(got[a:b] - ref[a:b]).max() / max(np.abs(ref[a:b]).max(), 1e-300))
    return np.array(errs)


def _solve(model, st, team, prec="fp64"):
    from paper_1609_06779_gb300 import fd
    cs = fd.ChainSet(model)
    b = fd.Batch(cs)
    dt = torch.float64 if prec == "fp64" else torch.float32
    t = lambda a: torch.tensor(a, dtype=dt, device="cuda")
    status = torch.full((b.n_problems,), -1, dtype=torch.int32, device="cuda")
    out = fd.solve(b, t(st.q), t(st.qdot), t(st.tau), algo="abia_scan", prec=prec, team=team,
                   status=status)
    torch.cuda.synchronize()
    return out.cpu().numpy(), status.cpu().numpy()


@pytest.mark.parametrize("team", [8, 16, 32, 64, 128, 256, 0])
def test_abia_scan_ragged_fp64(team):
    model = synth.random_chains([1, 2, 3, 5, 7, 8, 13, 31, 32, 33, 47, 64, 100, 0] * 2, seed=61)
    st = synth.random_states(model.n_links_total, seed=62)
    ref = oracle.fd(model, st.q, st.qdot, st.tau)
    aba = oracle.fd(model, st.q, st.qdot, st.tau, algo="aba")
    got, status = _solve(model, st, team)
    assert (status == 0).all()
    err = _rel_err(got, ref, model.offsets)
    floor = _rel_err(aba, ref, model.offsets)
    assert (err <= np.maximum(1e-10, 10 * floor)).all(), err.max()


@pytest.mark.parametrize("n,count,teams", [(256, 4, (32, 64, 256)), (1024, 2, (64, 256))])
def test_abia_scan_long_chains_fp64(n, count, teams):
    """The stability check: on long chains the scan's error stays at the oracle's
    own floor (its ABA route against its Cholesky route)."""
    model = synth.random_chains([n] * count, seed=n + 7)
    st = synth.random_states(model.n_links_total, seed=n + 8)
    ref = oracle.fd(model, st.q, st.qdot, st.tau, n_threads=8)
    aba = oracle.fd(model, st.q, st.qdot, st.tau, algo="aba", n_threads=8)
    floor = _rel_err(aba, ref, model.offsets)
    for team in teams:
        got, status = _solve(model, st, team)
        assert (status == 0).all(), team
        err = _rel_err(got, ref, model.offsets)
        print(f"n={n} team {team}: max err {err.max():.2e}, oracle floor {floor.max():.2e}")
        assert (err <= np.maximum(1e-10, 10 * floor)).all(), (team, err.max(), floor.max())


def test_abia_scan_unsupported_options():
    from paper_1609_06779_gb300 import fd
    model = synth.random_chains([8, 9], seed=3)
    st = synth.random_states(model.n_links_total, seed=4)
    with pytest.raises(fd.FDError) as e:
        _solve(model, st, 8, prec="fp32")
    assert e.value.status == 8
    with pytest.raises(fd.FDError):
        _solve(model, st, 4)       # teams of 8 .. 256
    cs = fd.ChainSet(model)
    b = fd.Batch(cs)
    x = torch.zeros(17, dtype=torch.float32, device="cuda")
    with pytest.raises(fd.FDError) as e:
        fd.adjoint(b, x, x, x, x, algo="abia_scan", prec="fp32")
    assert e.value.status == 8


@pytest.mark.parametrize("team", [8, 64])
def test_abia_scan_adjoint_matches_abia(team):
    """The adjoint with the scan's shared elimination (FD and M^-1 w in one pass,
    MODE_FD2) equals ABIA's within the FP64 bars (tau_bar = M^-1 w a plain solve;
    q_bar, qdot_bar the adjoint's 1e-6 bar against central differences)."""
    from paper_1609_06779_gb300 import fd
    model = synth.random_chains([1, 5, 12, 33, 64, 100], seed=71)
    st = synth.random_states(model.n_links_total, seed=72)
    cs = fd.ChainSet(model)
    b = fd.Batch(cs)
    t = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")
    w = torch.randn(model.n_links_total, dtype=torch.float64, device="cuda")
    q, qd, tau = t(st.q), t(st.qdot), t(st.tau)
    got = fd.adjoint(b, q, qd, tau, w, algo="abia_scan", team=team)
    ref = fd.adjoint(b, q, qd, tau, w, algo="abia", team=8)
    for x, y, tol in zip(got, ref, (1e-6, 1e-6, 1e-9, 1e-6)):
        err = _rel_err(x.cpu().numpy(), y.cpu().numpy(), model.offsets)
        assert err.max() < tol, (team, err.max())
    # and the forward result of the shared pass equals the plain solve's
    qdd_scan = fd.solve(b, q, qd, tau, algo="abia_scan", team=team).cpu().numpy()
    qdd = fd.solve(b, q, qd, tau, algo="abia").cpu().numpy()
    assert _rel_err(qdd_scan, qdd, model.offsets).max() < 1e-10
