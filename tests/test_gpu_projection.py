"""CFA with a general projection W (fd_solve_cfa_projected), called through the
C ABI: W_i = Wc_i Q_i with Q_i given per link or formed by block Jacobi
(Q_i = L_i^{-T}, D_i = L_i L_i^T). The paper's conclusion leaves the choice of W
in Eq. cfa-eq1 open; every admissible W gives the same qdd (Eq. cfa-eq2 is a
congruence of the same system), so the oracle here is the Cholesky route and
the oracle's CFA with the same W, and the checks that the projection is really
applied are that it changes the arithmetic (results not bit-equal to the
canonical CFA) without changing the result."""
import numpy as np
import pytest

import oracle
import oracle.dense as dense
from paper_1609_06779_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

RAGGED = [1, 2, 3, 5, 7, 8, 13, 31, 32, 33, 47, 64, 100]
EPS32 = float(np.finfo(np.float32).eps)


def _rel_err(got, ref, offsets):
    errs = []
    for p in range(len(offsets) - 1):
        a, b = offsets[p], offsets[p + 1]
        if b == a:
            continue
        scale = max(np.abs(ref[a:b]).max(), 1e-300)
        errs.append(np.abs(got[a:b] - ref[a:b]).max() / scale)
    return np.array(errs)


def _setup(model, st, prec):
    from paper_1609_06779_gb300 import fd
    cs = fd.ChainSet(model)
    b = fd.Batch(cs)
    dt = torch.float64 if prec == "fp64" else torch.float32
    q, qd, tau = (torch.tensor(x, dtype=dt, device="cuda") for x in (st.q, st.qdot, st.tau))
    return fd, b, q, qd, tau


def _given_w(model, seed):
    """W_i = (orthonormal complement of S_i) Z_i with Z_i random and invertible."""
    rng = np.random.default_rng(seed)
    _, Wb = dense.projection(model)
    Z = rng.standard_normal((model.n_links_total, 5, 5)) + 3 * np.eye(5)
    return Wb @ Z


def _solve(fd, b, q, qd, tau, proj, prec, team, Q=None):
    status = torch.full((b.n_problems,), -1, dtype=torch.int32, device="cuda")
    out = fd.solve_cfa_projected(b, q, qd, tau, projection=proj, Q=Q, prec=prec, team=team,
                                 status=status)
    torch.cuda.synchronize()
    return out, status.cpu().numpy()


@pytest.mark.parametrize("team", [1, 2, 8, 32, 128, 256, 0])
def test_projected_cfa_fp64_parity(team):
    model = synth.random_chains(RAGGED * 2, seed=21)
    st = synth.random_states(model.n_links_total, seed=22)
    ref = oracle.fd(model, st.q, st.qdot, st.tau, algo="cholesky")
    aba = oracle.fd(model, st.q, st.qdot, st.tau, algo="aba")
    W = _given_w(model, 23)
    cfa_w = oracle.fd_cfa_w(model, st.q, st.qdot, st.tau, W)
    # the oracle's own floor: its two routes' disagreement and its CFA with this W
    floor = np.maximum(_rel_err(aba, ref, model.offsets), _rel_err(cfa_w, ref, model.offsets))
    tol = np.maximum(1e-10, 10 * floor)
    fd, b, q, qd, tau = _setup(model, st, "fp64")
    Q = torch.tensor(fd.projection_to_canonical(model.axes, W), device="cuda").contiguous()
    canon, _ = _solve(fd, b, q, qd, tau, "canonical", "fp64", team)
    for proj, Qa in (("given", Q), ("block_jacobi", None)):
        out, status = _solve(fd, b, q, qd, tau, proj, "fp64", team, Qa)
        assert (status == 0).all(), proj
        err = _rel_err(out.cpu().numpy(), ref, model.offsets)
        assert (err <= tol).all(), (proj, err.max(), tol[np.argmax(err - tol)])
        # the projection is applied: other rounding, same result
        assert not torch.equal(out, canon), proj


def test_projected_canonical_is_the_cfa_kernel():
    model = synth.random_chains([32] * 40 + [7, 64, 1], seed=24)
    st = synth.random_states(model.n_links_total, seed=25)
    for prec in ("fp64", "fp32"):
        fd, b, q, qd, tau = _setup(model, st, prec)
        for team in (8, 32):
            ref = fd.solve(b, q, qd, tau, algo="cfa", prec=prec, team=team)
            out, status = _solve(fd, b, q, qd, tau, "canonical", prec, team)
            assert (status == 0).all()
            assert torch.equal(out, ref), (prec, team)


def _orthogonal_w(model, seed):
    """W_i = (orthonormal complement of S_i) Z_i with Z_i random orthogonal."""
    rng = np.random.default_rng(seed)
    _, Wb = dense.projection(model)
    Z = np.linalg.qr(rng.standard_normal((model.n_links_total, 5, 5)))[0]
    return Wb @ Z


def test_projected_cfa_fp32_bars():
    """FP32 with an orthonormal W (given) and with block Jacobi against the
    single-precision bars of the other FP32 paths: 1e-4 where cond(M) eps32 <=
    1e-4, everywhere max(1e-4, 4 cond(M) eps32). (A W whose Q_i are far from
    orthogonal multiplies the condition of the eliminated system by up to
    cond(Q_i)^2 and is not held to these bars.)"""
    model = synth.random_chains([1, 2, 4, 7, 8, 13, 32] * 6, seed=26)
    st = synth.random_states(model.n_links_total, seed=27)
    ref = oracle.fd(model, st.q, st.qdot, st.tau)
    cond = []
    for p in range(model.n_chains):
        a, z = model.offsets[p], model.offsets[p + 1]
        cond.append(np.linalg.cond(oracle.mass_matrix(model.chain(p), st.q[a:z])))
    cond = np.array(cond)
    good = cond * EPS32 <= 1e-4
    assert good.mean() > 0.5
    fd, b, q, qd, tau = _setup(model, st, "fp32")
    W = _orthogonal_w(model, 28)
    Q = torch.tensor(fd.projection_to_canonical(model.axes, W), device="cuda").contiguous()
    for proj, Qa in (("given", Q), ("block_jacobi", None)):
        for team in (1, 8):
            out, status = _solve(fd, b, q, qd, tau, proj, "fp32", team, Qa)
            assert (status == 0).all(), (proj, team)
            err = _rel_err(out.double().cpu().numpy(), ref, model.offsets)
            assert err[good].max() < 1e-4, (proj, team, err[good].max())
            bound = np.maximum(1e-4, 4 * cond * EPS32)
            assert (err <= bound).all(), (proj, team, (err / bound).max())


def test_projected_cfa_bad_arguments():
    model = synth.random_chains([5, 6], seed=29)
    st = synth.random_states(model.n_links_total, seed=30)
    fd, b, q, qd, tau = _setup(model, st, "fp64")
    lib = fd.load()
    out = torch.empty_like(q)
    ws = fd.workspace(b, "cfa", "fp64", 8)
    args = lambda prec, team, proj, Q: (b.handle, q.data_ptr(), qd.data_ptr(), tau.data_ptr(),
                                        out.data_ptr(), prec, team, proj, Q, ws.data_ptr(),
                                        ws.numel(), None, None)
    assert lib.fd_solve_cfa_projected(*args(2, 8, 2, None)) == 8   # mixed: unsupported
    assert lib.fd_solve_cfa_projected(*args(0, 8, 1, None)) == 1   # given without Q
    assert lib.fd_solve_cfa_projected(*args(0, 3, 2, None)) == 1   # team 3
    assert lib.fd_solve_cfa_projected(*args(0, 8, 7, None)) == 1   # unknown projection
    assert lib.fd_solve_cfa_projected(b.handle, q.data_ptr(), qd.data_ptr(), tau.data_ptr(),
                                      out.data_ptr(), 0, 8, 2, None, ws.data_ptr(), 16, None,
                                      None) == 1  # workspace too small
    with pytest.raises(fd.FDError):
        fd.solve_cfa_projected(b, q, qd, tau, projection="given", Q=None)
    with pytest.raises(fd.FDError):
        fd.solve_cfa_projected(b, q, qd, tau, projection="given",
                               Q=torch.zeros(7, dtype=torch.float64, device="cuda"))
    with pytest.raises(fd.FDError):
        fd.solve_cfa_projected(b, q, qd, tau, projection="bogus")
