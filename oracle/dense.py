"""Dense global-matrix definitions for tiny chains (FP64 numpy).

TEST INFRASTRUCTURE ONLY (see the package docstring). These routines write the
paper's global matrix equations out literally, with library dense solves as the
only steps, so that the C oracle's recursions can be checked against them:

* Eq. 2a-2d: (I - Gamma) V = S qd + c_V, (I - Gamma) Vd = S qdd - ad_{S qd}(Gamma V)
  + c_Vd, (I - Gamma)^T F = J Vd - ad_V^T (J V), tau = S^T F. The sign of the
  ad term is the reading in which it equals ad_{V_i}(S_i qd_i) link by link
  (Eq. 1 and Eq. 2b disagree on the sign convention of ad).
* Eq. 3 (definition after Eq. eq-motion): M(q) = S^T (I-Gamma)^{-T} J (I-Gamma)^{-1} S.
* Kinematic trees (beyond the paper's serial chains): the same equations with
  X_i in Gamma's block (i, parent(i)) and the base acceleration entering every
  link on the base.
* Eq. cfa-eq2 and Eq. fijany-final: T = (I-Gamma) J^{-1} (I-Gamma)^T,
  A = W^T T W, B = W^T T S, C = S^T T S, M^{-1} = C - B^T A^{-1} B.
"""
from __future__ import annotations

import numpy as np


def _skew(v):
    return np.array([[0.0, -v[2], v[1]], [v[2], 0.0, -v[0]], [-v[1], v[0], 0.0]])


def _rot(a, q):
    K = _skew(a)
    return np.eye(3) + np.sin(q) * K + (1.0 - np.cos(q)) * (K @ K)


def _Ad(R, p):
    A = np.zeros((6, 6))
    A[:3, :3] = R
    A[3:, 3:] = R
    A[3:, :3] = _skew(p) @ R
    return A


def _ad(V):
    A = np.zeros((6, 6))
    A[:3, :3] = _skew(V[:3])
    A[3:, 3:] = _skew(V[:3])
    A[3:, :3] = _skew(V[3:])
    return A


def link_operators(model, q):
    """Per link: X_i = Ad_{g_{i-1,i}(q_i)^{-1}} and S_i = (a_i; 0)."""
    n = model.axes.shape[0]
    X, S = [], []
    for i in range(n):
        fr = model.frames[i]
        R = fr[:9].reshape(3, 3) @ _rot(model.axes[i], q[i])
        p = fr[9:]
        X.append(_Ad(R.T, -R.T @ p))
        S.append(np.concatenate([model.axes[i], np.zeros(3)]))
    return X, S


def parent_of(model, i):
    """The link that link i's joint attaches to (-1: the base): i - 1 on a serial
    chain, ``model.parents[i]`` on a kinematic tree."""
    parents = getattr(model, "parents", None)
    return i - 1 if parents is None else int(parents[i])


def global_matrices(model, q):
    """Gamma (6n x 6n: X_i in block row i, column parent(i); the block sub-
    diagonal on a serial chain), S (6n x n), J (6n x 6n)."""
    n = model.axes.shape[0]
    X, S = link_operators(model, q)
    G = np.zeros((6 * n, 6 * n))
    Sg = np.zeros((6 * n, n))
    Jg = np.zeros((6 * n, 6 * n))
    for i in range(n):
        l = parent_of(model, i)
        if l >= 0:
            G[6 * i:6 * i + 6, 6 * l:6 * l + 6] = X[i]
        Sg[6 * i:6 * i + 6, i] = S[i]
        Jg[6 * i:6 * i + 6, 6 * i:6 * i + 6] = model.inertias[i].reshape(6, 6)
    return G, Sg, Jg, X


def mass_matrix(model, q):
    """Eq. 3's definition M = S^T (I-Gamma)^{-T} J (I-Gamma)^{-1} S."""
    G, S, J, _ = global_matrices(model, q)
    I = np.eye(G.shape[0])
    Y = np.linalg.solve(I - G, S)
    return Y.T @ J @ Y


def inverse_dynamics(model, q, qd, qdd, gravity=None):
    """Eq. 2a-2d as dense linear systems; the base terms enter the first block."""
    g = model.gravity if gravity is None else np.asarray(gravity)
    G, S, J, X = global_matrices(model, q)
    n = S.shape[1]
    I = np.eye(6 * n)
    V = np.linalg.solve(I - G, S @ qd)
    GV = G @ V
    Sqd = S @ qd
    adterm = np.zeros(6 * n)
    for i in range(n):
        adterm[6 * i:6 * i + 6] = -_ad(Sqd[6 * i:6 * i + 6]) @ GV[6 * i:6 * i + 6]
    c = np.zeros(6 * n)
    for i in range(n):  # every link on the base takes the base's acceleration (0; -g)
        if parent_of(model, i) < 0:
            c[6 * i:6 * i + 6] = X[i] @ np.concatenate([np.zeros(3), -g])
    Vd = np.linalg.solve(I - G, S @ qdd + adterm + c)
    rhs = J @ Vd
    for i in range(n):
        Vi = V[6 * i:6 * i + 6]
        Ji = J[6 * i:6 * i + 6, 6 * i:6 * i + 6]
        rhs[6 * i:6 * i + 6] -= _ad(Vi).T @ (Ji @ Vi)
    F = np.linalg.solve((I - G).T, rhs)
    return S.T @ F


def forward_dynamics(model, q, qd, tau):
    """qdd = M^{-1} (tau - ID(q, qd, 0)) with M and ID from the definitions above
    (Eq. 4), for a chain or a kinematic tree."""
    n = model.axes.shape[0]
    return np.linalg.solve(mass_matrix(model, q), tau - inverse_dynamics(model, q, qd, np.zeros(n)))


def projection(model, rng=None):
    """Block-diagonal W (6n x 5n) with W_i^T S_i = 0; random orthonormal W_i if
    ``rng`` is given, else a deterministic orthonormal complement."""
    n = model.axes.shape[0]
    W = np.zeros((6 * n, 5 * n))
    Wb = np.zeros((n, 6, 5))
    for i in range(n):
        a = model.axes[i]
        Q, _ = np.linalg.qr(np.column_stack([a, np.eye(3)]))
        b, c = Q[:, 1], Q[:, 2]
        Wi = np.zeros((6, 5))
        Wi[:3, 0], Wi[:3, 1] = b, c
        Wi[3:, 2:] = np.eye(3)
        if rng is not None:
            Z, _ = np.linalg.qr(rng.standard_normal((5, 5)))
            Wi = Wi @ Z
        W[6 * i:6 * i + 6, 5 * i:5 * i + 5] = Wi
        Wb[i] = Wi
    return W, Wb


def cfa_matrices(model, q, W=None):
    """T, A, B, C (Eq. cfa-eq2, Eq. fijany-final) with the given W (dense)."""
    G, S, J, _ = global_matrices(model, q)
    if W is None:
        W, _ = projection(model)
    I = np.eye(G.shape[0])
    T = (I - G) @ np.linalg.inv(J) @ (I - G).T
    return dict(T=T, A=W.T @ T @ W, B=W.T @ T @ S, C=S.T @ T @ S, W=W, S=S)


def fd_cfa(model, q, qd, tau, W=None):
    """qdd = C tau_d + B^T F_c with A F_c = -B tau_d (Eq. cfa-eq2, dense solve)."""
    m = cfa_matrices(model, q, W)
    td = tau - inverse_dynamics(model, q, qd, np.zeros_like(q))
    Fc = np.linalg.solve(m["A"], -m["B"] @ td)
    return m["C"] @ td + m["B"].T @ Fc


# ------------------------------------------------------ closed kinematic loops

def _pose(R, p):
    T = np.eye(4)
    T[:3, :3], T[:3, 3] = R, p
    return T


def world_poses(model, q):
    """Pose of every link frame in the base frame (4 x 4), by composing each
    link's home transform and joint rotation onto its parent's pose."""
    n = model.axes.shape[0]
    out = []
    for i in range(n):
        fr = model.frames[i]
        gi = _pose(fr[:9].reshape(3, 3) @ _rot(model.axes[i], q[i]), fr[9:])
        l = parent_of(model, i)
        out.append(gi if l < 0 else out[l] @ gi)
    return out


def _ancestors_or_self(model, i):
    path = []
    while i >= 0:
        path.append(i)
        i = parent_of(model, i)
    return path


def loop_constraints(model, q, qd, loops):
    """Constraint rows of revolute loop joints closing a tree (beyond the
    paper). Loop k joins frame F_a (pose loops["frame_a"][k] in link a's frame,
    a = -1: the base) and frame F_b (loops["frame_b"][k] in link b's frame) by a
    revolute joint about their x axes: the relative twist
    V_rel = V_Fb - Ad_{g_{Fb<-Fa}} V_Fa (body twist of F_b relative to F_a, in F_b
    coordinates) may only turn about x, so components 1..5 vanish. Returns G
    (5K x n) with V_rel[1..5] = G qd, and gamma (5K) = (dG/dt) qd, the velocity
    product of the constraint acceleration G qdd + gamma = 0, both from world
    quantities: with s_j = Ad_{g_0j} S_j (joint axes as world twists) and the
    links' world twists V^s_j = sum over j's path of s_i qd_i,
      V_rel = Ad_{g_0Fb^{-1}} (V^s_b - V^s_a),
      d/dt V_rel|_{qdd=0} = -ad_{V_Fb} V_rel + Ad_{g_0Fb^{-1}} sum +-ad_{V^s_j} s_j qd_j."""
    n = model.axes.shape[0]
    g0 = world_poses(model, q)
    s = []
    for j in range(n):
        R, p = g0[j][:3, :3], g0[j][:3, 3]
        w = R @ model.axes[j]
        s.append(np.concatenate([w, np.cross(p, w)]))
    Vs = [None] * n
    for j in range(n):
        l = parent_of(model, j)
        Vs[j] = (np.zeros(6) if l < 0 else Vs[l]) + s[j] * qd[j]
    K = len(loops["a"])
    G = np.zeros((5 * K, n))
    gamma = np.zeros(5 * K)
    for k in range(K):
        a, b = int(loops["a"][k]), int(loops["b"][k])
        Ta, Tb = loops["frame_a"][k], loops["frame_b"][k]
        gFb = g0[b] @ _pose(Tb[:9].reshape(3, 3), Tb[9:])
        Rb, pb = gFb[:3, :3], gFb[:3, 3]
        AdInv = _Ad(Rb.T, -Rb.T @ pb)
        Gf = np.zeros((6, n))
        drift = np.zeros(6)
        for sign, link in ((1.0, b), (-1.0, a)):
            for j in _ancestors_or_self(model, link):
                Gf[:, j] += sign * s[j]
                drift += sign * _ad(Vs[j]) @ s[j] * qd[j]
        Vb_s = Vs[b]
        Va_s = Vs[a] if a >= 0 else np.zeros(6)
        Vrel = AdInv @ (Vb_s - Va_s)
        VFb = AdInv @ Vb_s
        G[5 * k:5 * k + 5] = (AdInv @ Gf)[1:]
        gamma[5 * k:5 * k + 5] = (-_ad(VFb) @ Vrel + AdInv @ drift)[1:]
    return G, gamma


def forward_dynamics_looped(model, q, qd, tau, loops):
    """qdd of a tree closed by revolute loop joints: the KKT system
    M qdd + G^T lam = tau - ID(q, qd, 0), G qdd = -gamma, solved densely."""
    n = model.axes.shape[0]
    M = mass_matrix(model, q)
    f = tau - inverse_dynamics(model, q, qd, np.zeros(n))
    G, gamma = loop_constraints(model, q, qd, loops)
    m = G.shape[0]
    KKT = np.zeros((n + m, n + m))
    KKT[:n, :n], KKT[:n, n:], KKT[n:, :n] = M, G.T, G
    sol = np.linalg.solve(KKT, np.concatenate([f, -gamma]))
    return sol[:n]
