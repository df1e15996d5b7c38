"""Pins of the FP64 CPU oracle against facts that do not come from the oracle:
closed forms derived here by hand, the paper's dense global-matrix definitions,
conservation laws, and agreement of independent routes (Section II-C's three
factorisations of M^{-1} all give the same qdd)."""
import numpy as np
import pytest

import oracle
import oracle.dense as dense
import oracle.scan as scan
from paper_1609_06779_gb300 import synth

G0 = 9.81


def _single_chain(axes, frames, inertias, gravity=synth.GRAVITY):
    axes = np.asarray(axes, dtype=float)
    return synth.ChainModel(axes=axes, frames=np.asarray(frames, dtype=float),
                            inertias=np.asarray(inertias, dtype=float).reshape(-1, 36),
                            offsets=np.array([0, axes.shape[0]], dtype=np.int64),
                            gravity=np.asarray(gravity, dtype=float))


def _frame(R=np.eye(3), p=(0, 0, 0)):
    return np.concatenate([np.asarray(R, float).reshape(9), np.asarray(p, float)])


def _random_spd3(rng):
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    return Q @ np.diag(rng.uniform(0.01, 0.1, 3)) @ Q.T


def _com_of(J):
    m = J[5, 5]
    C = -J[3:, :3] / m
    return m, np.array([C[2, 1], C[0, 2], C[1, 0]])


# ---------------------------------------------------------------- closed forms

@pytest.mark.parametrize("seed", range(5))
def test_single_pendulum_closed_form(seed):
    """n = 1, axis y perpendicular to gravity: M = I_yy + m (cx^2 + cz^2) and the
    gravity torque m g (cx cos q + cz sin q) follow from the COM height
    z = -cx sin q + cz cos q (Lagrange). No velocity term for one fixed axis."""
    rng = np.random.default_rng(seed)
    m = rng.uniform(0.5, 5.0)
    c = rng.uniform(-0.3, 0.3, 3)
    Ic = _random_spd3(rng)
    J = synth.rigid_body_inertia(np.array(m), c, Ic)
    model = _single_chain([[0, 1, 0]], [_frame()], J)
    q, qd, tau = rng.uniform(-np.pi, np.pi, 1), rng.standard_normal(1), rng.standard_normal(1) * 10
    expect = (tau[0] + m * G0 * (c[0] * np.cos(q[0]) + c[2] * np.sin(q[0]))) / (
        Ic[1, 1] + m * (c[0] ** 2 + c[2] ** 2))
    for algo in ("cholesky", "aba", "cfa"):
        got = oracle.fd(model, q, qd, tau, algo=algo)
        assert got[0] == pytest.approx(expect, rel=1e-12, abs=1e-12), algo


def _planar_arm(rng):
    l1 = rng.uniform(0.2, 0.8)
    lc1, lc2 = rng.uniform(0.05, 0.5, 2)
    m1, m2 = rng.uniform(0.5, 5.0, 2)
    I1m, I2m = _random_spd3(rng), _random_spd3(rng)
    cy1, cy2 = rng.uniform(-0.1, 0.1, 2)          # offsets along the axis do not matter
    J1 = synth.rigid_body_inertia(np.array(m1), np.array([lc1, cy1, 0.0]), I1m)
    J2 = synth.rigid_body_inertia(np.array(m2), np.array([lc2, cy2, 0.0]), I2m)
    model = _single_chain([[0, 1, 0], [0, 1, 0]], [_frame(), _frame(p=(l1, 0, 0))],
                          np.stack([J1, J2]))
    return model, dict(l1=l1, lc1=lc1, lc2=lc2, m1=m1, m2=m2, I1=I1m[1, 1], I2=I2m[1, 1])


def _planar_closed_form(p, q, qd, tau):
    """Two-link arm, parallel axes y, links along x at q = 0. Kinetic energy gives
    M; Christoffel symbols of M give the velocity terms; the potential
    U = g (m1 z1 + m2 z2) with z1 = -lc1 sin q1, z2 = -l1 sin q1 - lc2 sin(q1 + q2)."""
    l1, lc1, lc2, m1, m2, I1, I2 = (p[k] for k in ("l1", "lc1", "lc2", "m1", "m2", "I1", "I2"))
    c2 = np.cos(q[1])
    M = np.array([[I1 + I2 + m1 * lc1**2 + m2 * (l1**2 + lc2**2 + 2 * l1 * lc2 * c2),
                   I2 + m2 * (lc2**2 + l1 * lc2 * c2)],
                  [I2 + m2 * (lc2**2 + l1 * lc2 * c2), I2 + m2 * lc2**2]])
    h = m2 * l1 * lc2 * np.sin(q[1])
    cor = np.array([-h * (2 * qd[0] * qd[1] + qd[1] ** 2), h * qd[0] ** 2])
    grav = np.array([-G0 * (m1 * lc1 * np.cos(q[0]) + m2 * (l1 * np.cos(q[0])
                                                           + lc2 * np.cos(q[0] + q[1]))),
                     -G0 * m2 * lc2 * np.cos(q[0] + q[1])])
    return M, np.linalg.solve(M, tau - cor - grav)


@pytest.mark.parametrize("seed", range(6))
def test_two_link_planar_arm_closed_form(seed):
    rng = np.random.default_rng(100 + seed)
    model, p = _planar_arm(rng)
    q = rng.uniform(-np.pi, np.pi, 2)
    qd = rng.standard_normal(2) * 2
    tau = rng.standard_normal(2) * 10
    M_cf, qdd_cf = _planar_closed_form(p, q, qd, tau)
    np.testing.assert_allclose(oracle.mass_matrix(model, q), M_cf, rtol=1e-12, atol=1e-13)
    for algo in ("cholesky", "aba", "cfa"):
        np.testing.assert_allclose(oracle.fd(model, q, qd, tau, algo=algo), qdd_cf,
                                   rtol=1e-11, atol=1e-11, err_msg=algo)


# ------------------------------------------------------- definitions and routes

@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (3, 2), (5, 3), (8, 4)])
def test_mass_matrix_matches_dense_definition(n, seed):
    model = synth.random_chains(n, seed=seed, random_home_rotation=True)
    st = synth.random_states(n, seed=seed + 50)
    M = oracle.mass_matrix(model, st.q)
    np.testing.assert_allclose(M, dense.mass_matrix(model, st.q), rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(M, M.T, rtol=0, atol=1e-13 * np.abs(M).max())
    assert np.linalg.eigvalsh(M).min() > 0


@pytest.mark.parametrize("n,seed", [(1, 0), (3, 2), (6, 3), (9, 4)])
def test_inverse_dynamics_matches_dense_equations(n, seed):
    model = synth.random_chains(n, seed=seed, random_home_rotation=True)
    st = synth.random_states(n, seed=seed + 7)
    qdd = np.random.default_rng(seed).standard_normal(n)
    np.testing.assert_allclose(oracle.rnea(model, st.q, st.qdot, qdd),
                               dense.inverse_dynamics(model, st.q, st.qdot, qdd),
                               rtol=1e-11, atol=1e-11)


@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (7, 2), (16, 3), (33, 4)])
def test_three_factorisations_agree_and_residual(n, seed):
    model = synth.random_chains(n, seed=seed)
    st = synth.random_states(n, seed=seed + 1)
    ref = oracle.fd(model, st.q, st.qdot, st.tau, algo="cholesky")
    M = oracle.mass_matrix(model, st.q)
    tol = 1e-15 * np.linalg.cond(M) * 50
    scale = max(np.abs(ref).max(), 1.0)
    for algo in ("aba", "cfa"):
        got = oracle.fd(model, st.q, st.qdot, st.tau, algo=algo)
        assert np.abs(got - ref).max() / scale < tol, algo
    # residual of the inverse dynamics at the solution: ID(q, qd, qdd) = tau
    res = oracle.rnea(model, st.q, st.qdot, ref) - st.tau
    assert np.abs(res).max() < 1e-13 * np.abs(M).max() * max(np.abs(ref).max(), 1.0) * n


def test_zero_state_no_gravity_is_inverse_inertia():
    n = 6
    model = synth.random_chains(n, seed=11, gravity=[0.0, 0.0, 0.0])
    st = synth.random_states(n, seed=12)
    M = oracle.mass_matrix(model, st.q)
    expect = np.linalg.solve(M, st.tau)
    for algo in ("cholesky", "aba", "cfa"):
        np.testing.assert_allclose(oracle.fd(model, st.q, np.zeros(n), st.tau, algo=algo),
                                   expect, rtol=1e-10, atol=1e-12)


def _rotate_frames(model, rng):
    """Re-express every child frame by a random rotation Q_i (frame i' = i Q_i)."""
    n = model.axes.shape[0]
    Qs = [np.linalg.qr(rng.standard_normal((3, 3)))[0] for _ in range(n)]
    Qs = [Q if np.linalg.det(Q) > 0 else -Q for Q in Qs]
    axes = np.empty_like(model.axes)
    frames = np.empty_like(model.frames)
    J = np.empty_like(model.inertias)
    for i in range(n):
        Qp = Qs[i - 1] if i > 0 else np.eye(3)
        Q = Qs[i]
        R0 = model.frames[i, :9].reshape(3, 3)
        p0 = model.frames[i, 9:]
        axes[i] = Q.T @ model.axes[i]
        frames[i, :9] = (Qp.T @ R0 @ Q).reshape(9)
        frames[i, 9:] = Qp.T @ p0
        B = np.zeros((6, 6)); B[:3, :3] = Q; B[3:, 3:] = Q
        J[i] = (B.T @ model.inertias[i].reshape(6, 6) @ B).reshape(36)
    return synth.ChainModel(axes, frames, J, model.offsets.copy(), model.gravity.copy())


@pytest.mark.parametrize("seed", range(3))
def test_link_frame_invariance(seed):
    """qdd does not depend on how each link frame is oriented (coordinate-free
    notation of Section II)."""
    rng = np.random.default_rng(seed)
    model = synth.random_chains(7, seed=seed, random_home_rotation=True)
    st = synth.random_states(7, seed=seed + 3)
    rot = _rotate_frames(model, rng)
    for algo in ("cholesky", "aba", "cfa"):
        np.testing.assert_allclose(oracle.fd(rot, st.q, st.qdot, st.tau, algo=algo),
                                   oracle.fd(model, st.q, st.qdot, st.tau, algo=algo),
                                   rtol=1e-9, atol=1e-9)


# ------------------------------------------------------------ energy and power

def _potential(model, q):
    """U = -sum_i m_i g . com_i, world COMs by forward kinematics written here."""
    R, p = np.eye(3), np.zeros(3)
    U = 0.0
    for i in range(model.axes.shape[0]):
        a = model.axes[i]
        K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
        Rq = np.eye(3) + np.sin(q[i]) * K + (1 - np.cos(q[i])) * K @ K
        R0 = model.frames[i, :9].reshape(3, 3)
        p = p + R @ model.frames[i, 9:]
        R = R @ R0 @ Rq
        m, c = _com_of(model.inertias[i].reshape(6, 6))
        U -= m * model.gravity @ (p + R @ c)
    return U


def _energy(model, q, qd):
    return 0.5 * qd @ oracle.mass_matrix(model, q) @ qd + _potential(model, q)


@pytest.mark.parametrize("n,seed", [(2, 0), (5, 1), (9, 2)])
def test_power_balance(n, seed):
    """qd . tau_bias = 1/2 qd^T dM/dt qd + dU/dt (central differences along qd):
    the velocity and gravity terms of the bias torque do no net work beyond the
    change of kinetic and potential energy."""
    model = synth.random_chains(n, seed=seed)
    st = synth.random_states(n, seed=seed + 9)
    q, qd = st.q, st.qdot
    bias = oracle.rnea(model, q, qd)
    h = 1e-6
    dM = (oracle.mass_matrix(model, q + h * qd) - oracle.mass_matrix(model, q - h * qd)) / (2 * h)
    dU = (_potential(model, q + h * qd) - _potential(model, q - h * qd)) / (2 * h)
    lhs = qd @ bias
    rhs = 0.5 * qd @ dM @ qd + dU
    assert lhs == pytest.approx(rhs, rel=1e-6, abs=1e-6)


def _rk4_energy_drift(model, q, qd, dt, T):
    f = lambda q_, v_: oracle.fd(model, q_, v_, np.zeros_like(q_))
    E0 = _energy(model, q, qd)
    for _ in range(int(round(T / dt))):
        k1q, k1v = qd, f(q, qd)
        k2q, k2v = qd + 0.5 * dt * k1v, f(q + 0.5 * dt * k1q, qd + 0.5 * dt * k1v)
        k3q, k3v = qd + 0.5 * dt * k2v, f(q + 0.5 * dt * k2q, qd + 0.5 * dt * k2v)
        k4q, k4v = qd + dt * k3v, f(q + dt * k3q, qd + dt * k3v)
        q = q + dt / 6 * (k1q + 2 * k2q + 2 * k3q + k4q)
        qd = qd + dt / 6 * (k1v + 2 * k2v + 2 * k3v + k4v)
    return abs(_energy(model, q, qd) - E0) / abs(E0)


@pytest.mark.parametrize("n", [2, 5])
def test_zero_torque_energy_conservation(n):
    model = synth.random_chains(n, seed=21 + n)
    st = synth.random_states(n, seed=5)
    q, qd = st.q, st.qdot * 0.5
    d1 = _rk4_energy_drift(model, q, qd, 2e-4, 0.1)
    d2 = _rk4_energy_drift(model, q, qd, 1e-4, 0.1)
    assert d2 < 1e-8
    # fourth-order integrator: halving dt cuts the drift by about 16
    assert d2 < d1 / 8 or d1 < 1e-12


# ------------------------------------------------------------------------ CFA

@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (5, 2), (8, 3)])
def test_cfa_blocks_and_schur_identity(n, seed):
    model = synth.random_chains(n, seed=seed, random_home_rotation=True)
    st = synth.random_states(n, seed=seed + 2)
    blk = oracle.cfa_blocks(model, st.q)
    W = np.zeros((6 * n, 5 * n))
    for i in range(n):
        W[6 * i:6 * i + 6, 5 * i:5 * i + 5] = blk["W"][i]
    mats = dense.cfa_matrices(model, st.q, W)
    A, B, C, S = mats["A"], mats["B"], mats["C"], mats["S"]
    # W^T S = 0 (Eq. cfa-eq1)
    assert np.abs(W.T @ S).max() < 1e-14
    # A block tri-diagonal, symmetric, lower blocks = U^T (Eq. A_mat), SPD
    for i in range(n):
        for j in range(n):
            blkA = A[5 * i:5 * i + 5, 5 * j:5 * j + 5]
            if abs(i - j) > 1:
                assert np.abs(blkA).max() < 1e-12
        np.testing.assert_allclose(blk["D"][i], A[5 * i:5 * i + 5, 5 * i:5 * i + 5],
                                   rtol=1e-12, atol=1e-12)
        if i + 1 < n:
            np.testing.assert_allclose(blk["U"][i], A[5 * i:5 * i + 5, 5 * i + 5:5 * i + 10],
                                       rtol=1e-12, atol=1e-12)
            np.testing.assert_allclose(blk["U"][i].T, A[5 * i + 5:5 * i + 10, 5 * i:5 * i + 5],
                                       rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(blk["D"][i], blk["D"][i].T, atol=1e-12)
    assert np.linalg.eigvalsh(A).min() > 0
    # B and C blocks (C tri-diagonal)
    for i in range(n):
        for k, j in enumerate((i - 1, i, i + 1)):
            if 0 <= j < n:
                np.testing.assert_allclose(blk["B"][i, k], B[5 * i:5 * i + 5, j],
                                           rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(blk["Cd"][i], C[i, i], rtol=1e-12)
        if i + 1 < n:
            np.testing.assert_allclose(blk["Co"][i], C[i, i + 1], rtol=1e-12, atol=1e-13)
    # M^{-1} = C - B^T A^{-1} B (Eq. fijany-final)
    M = oracle.mass_matrix(model, st.q)
    np.testing.assert_allclose(C - B.T @ np.linalg.solve(A, B), np.linalg.inv(M),
                               rtol=1e-9, atol=1e-9 * np.abs(np.linalg.inv(M)).max())


@pytest.mark.parametrize("seed", range(3))
def test_cfa_invariant_under_choice_of_w(seed):
    """qdd does not depend on the basis W_i of each joint's constraint space
    (Section III-B); F_c does."""
    n = 6
    rng = np.random.default_rng(seed)
    model = synth.random_chains(n, seed=seed)
    st = synth.random_states(n, seed=seed + 4)
    W1, _ = dense.projection(model)
    W2, _ = dense.projection(model, rng)
    a = dense.fd_cfa(model, st.q, st.qdot, st.tau, W1)
    b = dense.fd_cfa(model, st.q, st.qdot, st.tau, W2)
    c = oracle.fd(model, st.q, st.qdot, st.tau, algo="cfa")
    np.testing.assert_allclose(a, b, rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(a, c, rtol=1e-9, atol=1e-9)


@pytest.mark.parametrize("seed", range(3))
def test_cfa_with_given_w_matches_dense_solve(seed):
    """The oracle's CFA with a given, non-orthogonal W_i (Eq. cfa-eq1): its
    constraint-force coordinates F_c, which depend on W, equal the dense solve
    A F_c = -B tau_delta of Eq. cfa-eq2 with the same W; F_c(W_i Z_i) = Z_i^{-1}
    F_c(W_i); qdd equals the Cholesky route's. Two chains packed, so that the
    per-chain slicing is pinned too."""
    rng = np.random.default_rng(seed)
    lengths = [5, 3]
    model = synth.random_chains(lengths, seed=seed, random_home_rotation=True)
    st = synth.random_states(model.n_links_total, seed=seed + 7)
    _, Wb = dense.projection(model)
    Z = rng.standard_normal((model.n_links_total, 5, 5)) + 3 * np.eye(5)
    Wz = Wb @ Z
    qdd0, fc0 = oracle.fd_cfa_w(model, st.q, st.qdot, st.tau, Wb, return_fc=True)
    qdd1, fc1 = oracle.fd_cfa_w(model, st.q, st.qdot, st.tau, Wz, return_fc=True)
    ref = oracle.fd(model, st.q, st.qdot, st.tau, algo="cholesky")
    np.testing.assert_allclose(qdd0, ref, rtol=1e-9, atol=1e-9 * np.abs(ref).max())
    np.testing.assert_allclose(qdd1, ref, rtol=1e-9, atol=1e-9 * np.abs(ref).max())
    for i in range(model.n_links_total):
        np.testing.assert_allclose(fc1[i], np.linalg.solve(Z[i], fc0[i]), rtol=1e-8,
                                   atol=1e-8 * np.abs(fc0).max())
    # the dense solve, chain by chain
    for p in range(len(lengths)):
        a, z = int(model.offsets[p]), int(model.offsets[p + 1])
        one = _chain_of(model, a, z)
        n = z - a
        W = np.zeros((6 * n, 5 * n))
        for i in range(n):
            W[6 * i:6 * i + 6, 5 * i:5 * i + 5] = Wz[a + i]
        m = dense.cfa_matrices(one, st.q[a:z], W)
        td = st.tau[a:z] - dense.inverse_dynamics(one, st.q[a:z], st.qdot[a:z], np.zeros(n))
        fcd = np.linalg.solve(m["A"], -m["B"] @ td).reshape(n, 5)
        np.testing.assert_allclose(fc1[a:z], fcd, rtol=1e-8, atol=1e-8 * np.abs(fcd).max())
    # a W that is not a complement of S (W^T S != 0) changes qdd: W is used
    Wbad = Wz.copy()
    Wbad[:, :3, 0] += np.asarray(model.axes)[:, :]
    qbad = oracle.fd_cfa_w(model, st.q, st.qdot, st.tau, Wbad)
    assert np.abs(qbad - ref).max() > 1e-6 * np.abs(ref).max()


def _chain_of(model, a, z):
    """Links a .. z-1 of a packed model as a model of one chain."""
    return _single_chain(np.asarray(model.axes)[a:z], np.asarray(model.frames)[a:z],
                         np.asarray(model.inertias)[a:z], model.gravity)


def _random_btd(n, b, rng):
    """A random SPD symmetric block tri-diagonal system: A = L L^T with L block
    lower bi-diagonal."""
    Ld = [np.tril(rng.standard_normal((b, b))) + 3 * np.eye(b) for _ in range(n)]
    Ll = [rng.standard_normal((b, b)) for _ in range(n)]
    D = np.empty((n, b, b)); U = np.zeros((n, b, b))
    for i in range(n):
        D[i] = Ld[i] @ Ld[i].T + (Ll[i] @ Ll[i].T if i > 0 else 0)
        if i + 1 < n:
            U[i] = Ld[i] @ Ll[i + 1].T
    return D, U


def _dense_btd(D, U):
    n, b, _ = D.shape
    A = np.zeros((n * b, n * b))
    for i in range(n):
        A[b * i:b * i + b, b * i:b * i + b] = D[i]
        if i + 1 < n:
            A[b * i:b * i + b, b * i + b:b * i + 2 * b] = U[i]
            A[b * i + b:b * i + 2 * b, b * i:b * i + b] = U[i].T
    return A


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 7, 8, 9, 13, 16, 17, 31, 33])
def test_oee_matches_dense_solve(n):
    rng = np.random.default_rng(n)
    D, U = _random_btd(n, 5, rng)
    assert np.abs(U[n - 1]).max() == 0
    R = rng.standard_normal((n, 5))
    F, Df, Uf, _ = oracle.oee_solve(D, U, R)
    A = _dense_btd(D, U)
    x = np.linalg.solve(A, R.reshape(-1)).reshape(n, 5)
    # forward-error bound of a backward-stable solve: about cond(A) * eps
    err = np.abs(F - x).max() / np.abs(x).max()
    assert err < 50 * np.finfo(float).eps * np.linalg.cond(A)
    assert np.abs(Uf).max() == 0.0
    # every final diagonal block is SPD (each level is a Schur complement)
    for i in range(n):
        assert np.linalg.eigvalsh(0.5 * (Df[i] + Df[i].T)).min() > 0


def test_oee_level_count_and_schur_blocks():
    """After level 1 the even rows hold the Schur complement of A onto the even
    rows (odd rows eliminated), which is the cyclic-reduction system."""
    n, b = 8, 3
    rng = np.random.default_rng(7)
    D, U = _random_btd(n, b, rng)
    A = _dense_btd(D, U)
    # one level by hand through the oracle: solve with n=2 trick is not exposed, so
    # compare the final D of a 2-row system with its exact Schur complements
    D2, U2 = D[:2].copy(), U[:2].copy()
    U2[1] = 0
    R = rng.standard_normal((2, b))
    F, Df, _, _ = oracle.oee_solve(D2, U2, R)
    A2 = _dense_btd(D2, U2)
    S0 = D2[0] - U2[0] @ np.linalg.solve(D2[1], U2[0].T)
    S1 = D2[1] - U2[0].T @ np.linalg.solve(D2[0], U2[0])
    np.testing.assert_allclose(Df[0], S0, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(Df[1], S1, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(F.reshape(-1), np.linalg.solve(A2, R.reshape(-1)), rtol=1e-11)
    del A


# ------------------------------------------------------------------------ scan

@pytest.mark.parametrize("n", [1, 2, 3, 8, 13, 32])
def test_scan_equals_serial_recursion(n):
    rng = np.random.default_rng(n)
    b = rng.standard_normal((max(n - 1, 0), 6, 6)) * 0.4
    c = rng.standard_normal((n, 6))
    x = scan.serial_recursion(b, c)
    np.testing.assert_allclose(scan.solve_by_scan(b, c, "serial"), x, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(scan.solve_by_scan(b, c, "tree"), x, rtol=1e-11, atol=1e-11)
    # the bi-diagonal system itself: rows x_i - b_{i-1} x_{i-1} = c_i
    for i in range(1, n):
        np.testing.assert_allclose(x[i] - b[i - 1] @ x[i - 1], c[i], atol=1e-12)


def test_scan_operator_is_associative():
    rng = np.random.default_rng(3)
    a = scan.operators(rng.standard_normal((2, 6, 6)), rng.standard_normal((3, 6)))
    l = scan.combine(scan.combine(a[0], a[1]), a[2])
    r = scan.combine(a[0], scan.combine(a[1], a[2]))
    np.testing.assert_allclose(l, r, rtol=1e-12, atol=1e-12)


# ---------------------------------------------------------------- batch plumbing

def test_batch_and_shared_model_layouts():
    model = synth.random_chains([3, 1, 5, 2], seed=4)
    st = synth.random_states(model.n_links_total, seed=5)
    full = oracle.fd(model, st.q, st.qdot, st.tau, algo="cfa")
    for k in range(model.n_chains):
        a, b = model.offsets[k], model.offsets[k + 1]
        one = oracle.fd(model.chain(k), st.q[a:b], st.qdot[a:b], st.tau[a:b], algo="aba")
        np.testing.assert_allclose(full[a:b], one, rtol=1e-10, atol=1e-10)
    sub = oracle.fd(model, st.q, st.qdot, st.tau, algo="cholesky", problems=[2, 0])
    np.testing.assert_allclose(sub[:3], full[:3], rtol=1e-10)
    np.testing.assert_allclose(sub[4:9], full[4:9], rtol=1e-10)
    assert np.isnan(sub[3]) and np.isnan(sub[9:]).all()
    # shared model: every problem uses chain 0
    one = model.chain(2)
    ci, so = synth.replicate_model(one, 4)
    s2 = synth.random_states(20, seed=6)
    out = oracle.fd(one, s2.q, s2.qdot, s2.tau, algo="aba", chain_index=ci, state_offsets=so,
                    n_threads=2)
    for p in range(4):
        sl = slice(5 * p, 5 * p + 5)
        np.testing.assert_allclose(out[sl], oracle.fd(one, s2.q[sl], s2.qdot[sl], s2.tau[sl]),
                                   rtol=1e-10)


# ------------------------------------------------------------ kinematic trees

def _tree_world(model, q):
    """World rotation and position of every link of one tree by forward
    kinematics over the parent array, written here."""
    n = model.axes.shape[0]
    Rw, pw = [None] * n, [None] * n
    for i in range(n):
        a = model.axes[i]
        K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
        Rq = np.eye(3) + np.sin(q[i]) * K + (1 - np.cos(q[i])) * K @ K
        R0 = model.frames[i, :9].reshape(3, 3)
        l = int(model.parents[i])
        Rl, pl = (np.eye(3), np.zeros(3)) if l < 0 else (Rw[l], pw[l])
        pw[i] = pl + Rl @ model.frames[i, 9:]
        Rw[i] = Rl @ R0 @ Rq
    return Rw, pw


def _tree_potential(model, q):
    Rw, pw = _tree_world(model, q)
    U = 0.0
    for i in range(model.axes.shape[0]):
        m, c = _com_of(model.inertias[i].reshape(6, 6))
        U -= m * model.gravity @ (pw[i] + Rw[i] @ c)
    return U


def _tree_kinetic(model, q, qd):
    """1/2 sum V_i^T J_i V_i with each link's twist (omega; v) in its own frame
    from the world velocities of forward kinematics (omega_i = omega_parent +
    R_i a_i qd_i, v of the frame origin by the rigid-body transport)."""
    Rw, pw = _tree_world(model, q)
    n = model.axes.shape[0]
    w_w, v_w = [None] * n, [None] * n
    T = 0.0
    for i in range(n):
        l = int(model.parents[i])
        wl, vl, pl = (np.zeros(3), np.zeros(3), np.zeros(3)) if l < 0 else (w_w[l], v_w[l], pw[l])
        w_w[i] = wl + Rw[i] @ model.axes[i] * qd[i]
        v_w[i] = vl + np.cross(wl, pw[i] - pl)   # the joint sits at the link origin
        V = np.concatenate([Rw[i].T @ w_w[i], Rw[i].T @ v_w[i]])
        T += 0.5 * V @ model.inertias[i].reshape(6, 6) @ V
    return T


@pytest.mark.parametrize("seed", range(3))
def test_tree_chain_special_case(seed):
    """parents = i - 1 is the serial chain: the tree definitions reproduce the
    chain oracle's recursions (inverse dynamics, forward dynamics)."""
    model = synth.random_chains([6, 4], seed=seed, random_home_rotation=True)
    st = synth.random_states(model.n_links_total, seed=seed + 3)
    tree = synth.random_chains([6, 4], seed=seed, random_home_rotation=True)
    tree.parents = np.concatenate([np.arange(n) - 1 for n in tree.lengths()]).astype(np.int32)
    np.testing.assert_allclose(oracle.fd_tree(tree, st.q, st.qdot, st.tau),
                               oracle.fd(model, st.q, st.qdot, st.tau), rtol=1e-9, atol=1e-9)
    qdd = np.random.default_rng(seed).standard_normal(model.n_links_total)
    ref = np.concatenate([oracle.rnea(model.chain(p), st.q[a:z], st.qdot[a:z], qdd[a:z])
                          for p, (a, z) in enumerate(zip(model.offsets[:-1], model.offsets[1:]))])
    np.testing.assert_allclose(oracle.rnea_tree(tree, st.q, st.qdot, qdd), ref, rtol=1e-10,
                               atol=1e-10 * np.abs(ref).max())


def test_tree_of_two_branches_on_the_base_is_two_chains():
    """Two serial branches both on the base are two independent chains: M is
    block diagonal with the chains' mass matrices, qdd the chains' results."""
    c = synth.random_chains([4, 3], seed=9)
    st = synth.random_states(7, seed=10)
    tree = synth.ChainModel(c.axes, c.frames, c.inertias, np.array([0, 7], dtype=np.int64),
                            c.gravity, np.array([-1, 0, 1, 2, -1, 4, 5], dtype=np.int32))
    M = dense.mass_matrix(tree, st.q)
    np.testing.assert_allclose(M[:4, :4], oracle.mass_matrix(c.chain(0), st.q[:4]), rtol=1e-10)
    np.testing.assert_allclose(M[4:, 4:], oracle.mass_matrix(c.chain(1), st.q[4:]), rtol=1e-10)
    assert np.abs(M[:4, 4:]).max() == 0.0
    np.testing.assert_allclose(oracle.fd_tree(tree, st.q, st.qdot, st.tau),
                               oracle.fd(c, st.q, st.qdot, st.tau), rtol=1e-9, atol=1e-9)


@pytest.mark.parametrize("seed", range(3))
def test_tree_mass_matrix_is_kinetic_energy(seed):
    """1/2 qd^T M qd equals the kinetic energy of the links' twists from forward
    kinematics over the parent array; M is symmetric positive definite and
    zero between links on different paths to the base."""
    tree = synth.random_trees([12], seed=seed, random_home_rotation=True)
    assert len(set(tree.parents.tolist())) < 12  # it branches
    st = synth.random_states(12, seed=seed + 5)
    M = dense.mass_matrix(tree, st.q)
    np.testing.assert_allclose(0.5 * st.qdot @ M @ st.qdot, _tree_kinetic(tree, st.q, st.qdot),
                               rtol=1e-10)
    np.testing.assert_allclose(M, M.T, atol=1e-12)
    assert np.linalg.eigvalsh(M).min() > 0
    anc = [set() for _ in range(12)]
    for i in range(12):
        l = int(tree.parents[i])
        anc[i] = ({l} | anc[l]) if l >= 0 else set()
    for i in range(12):
        for j in range(12):
            if i != j and j not in anc[i] and i not in anc[j]:
                assert M[i, j] == 0.0


@pytest.mark.parametrize("seed", range(3))
def test_tree_power_balance(seed):
    """qd . tau_bias = 1/2 qd^T dM/dt qd + dU/dt on a tree, U by forward
    kinematics over the parent array (central differences along qd)."""
    tree = synth.random_trees([9], seed=seed + 4)
    st = synth.random_states(9, seed=seed + 11)
    q, qd = st.q, st.qdot
    bias = oracle.rnea_tree(tree, q, qd, np.zeros(9))
    h = 1e-6
    dM = (dense.mass_matrix(tree, q + h * qd) - dense.mass_matrix(tree, q - h * qd)) / (2 * h)
    dU = (_tree_potential(tree, q + h * qd) - _tree_potential(tree, q - h * qd)) / (2 * h)
    assert qd @ bias == pytest.approx(0.5 * qd @ dM @ qd + dU, rel=1e-6, abs=1e-6)
    # gravity alone: the bias at rest is the gradient of U
    g = oracle.rnea_tree(tree, q, np.zeros(9), np.zeros(9))
    grad = np.array([(_tree_potential(tree, q + h * e) - _tree_potential(tree, q - h * e)) / (2 * h)
                     for e in np.eye(9)])
    np.testing.assert_allclose(g, grad, rtol=1e-6, atol=1e-6)


# ------------------------------------------------------ closed kinematic loops

def _loop_setup(seed, n=24):
    tree = synth.random_trees([n], seed=seed, random_home_rotation=True)
    loops = synth.random_loops(tree, per_tree=2, seed=seed + 1)
    st = synth.random_states(n, seed=seed + 2)
    return tree, loops, st


def _rel_pose(model, q, loops, k):
    """h = g_0Fa^-1 g_0Fb of loop k, by forward kinematics written here."""
    Rw, pw = _tree_world(model, q)
    def frame(link, T):
        R0, p0 = (np.eye(3), np.zeros(3)) if link < 0 else (Rw[link], pw[link])
        H = np.eye(4)
        H[:3, :3] = R0 @ T[:9].reshape(3, 3)
        H[:3, 3] = p0 + R0 @ T[9:]
        return H
    Ha = frame(int(loops["a"][k]), loops["frame_a"][k])
    Hb = frame(int(loops["b"][k]), loops["frame_b"][k])
    return np.linalg.inv(Ha) @ Hb


def _twist_of(H):
    """The twist (omega; v) whose exponential is the small motion H."""
    from scipy.linalg import logm
    X = np.real(logm(H))
    return np.array([X[2, 1], X[0, 2], X[1, 0], X[0, 3], X[1, 3], X[2, 3]])


@pytest.mark.parametrize("seed", range(3))
def test_loop_constraint_rows_are_the_relative_motion(seed):
    """G's rows are components 1..5 of the body twist of F_b relative to F_a:
    central differences of the relative pose along each joint (forward
    kinematics written in the test) give its columns; gamma = (dG/dt) qd by
    central differences of G along qd."""
    tree, loops, st = _loop_setup(seed)
    G, gamma = dense.loop_constraints(tree, st.q, st.qdot, loops)
    h = 1e-6
    for k in range(len(loops["a"])):
        for j in range(tree.axes.shape[0]):
            e = np.zeros_like(st.q); e[j] = h
            H = np.linalg.inv(_rel_pose(tree, st.q - e, loops, k)) @ _rel_pose(tree, st.q + e, loops, k)
            col = _twist_of(H) / (2 * h)
            np.testing.assert_allclose(G[5 * k:5 * k + 5, j], col[1:], atol=1e-6)
    h = 1e-5
    Gp, _ = dense.loop_constraints(tree, st.q + h * st.qdot, st.qdot, loops)
    Gm, _ = dense.loop_constraints(tree, st.q - h * st.qdot, st.qdot, loops)
    np.testing.assert_allclose(gamma, (Gp - Gm) @ st.qdot / (2 * h), rtol=1e-6,
                               atol=1e-7 * np.abs(gamma).max())


@pytest.mark.parametrize("seed", range(3))
def test_looped_dynamics_satisfy_the_constraints(seed):
    """The KKT solution accelerates along the loops (G qdd = -gamma), its joint
    torques differ from the open tree's only by constraint forces (M qdd - (tau -
    bias) lies in the range of G^T), and without loops it is the tree's."""
    tree, loops, st = _loop_setup(seed)
    qdd = oracle.fd_looped(tree, st.q, st.qdot, st.tau,
                           dict(loops, tree=np.zeros(len(loops["a"]), dtype=np.int32)))
    G, gamma = dense.loop_constraints(tree, st.q, st.qdot, loops)
    np.testing.assert_allclose(G @ qdd, -gamma, atol=1e-9 * max(np.abs(gamma).max(), 1))
    M = dense.mass_matrix(tree, st.q)
    r = M @ qdd - (st.tau - oracle.rnea_tree(tree, st.q, st.qdot, np.zeros_like(st.q)))
    lam, *_ = np.linalg.lstsq(G.T, r, rcond=None)
    np.testing.assert_allclose(G.T @ lam, r, atol=1e-8 * np.abs(r).max())
    none = {k: v[:0] for k, v in loops.items()}
    np.testing.assert_allclose(oracle.fd_looped(tree, st.q, st.qdot, st.tau, none),
                               oracle.fd_tree(tree, st.q, st.qdot, st.tau), rtol=1e-12, atol=1e-12)
