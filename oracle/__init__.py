"""FP64 CPU oracle for forward dynamics of serial chains (arXiv 1609.06779).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only code that may import this package.
It shares no code with the CUDA path and never imports it.

* ``fd_oracle.c`` (compiled by :func:`build` with gcc) holds the per-chain
  recursions: inverse dynamics (Eq. 2a-2d), the mass matrix by JSIIA columns
  (Section II-C), FD by dense Cholesky (Eq. 4), ABIA (Section II-C) and CFA with
  odd-even elimination (Algorithms 1 and 2).
* ``dense.py`` writes the global-matrix definitions out densely for tiny chains
  (the mass matrix of Eq. 3's definition, T, A, B, C of Eq. cfa-eq2 and
  Eq. fijany-final).
* ``scan.py`` holds the scan formulation of a bi-diagonal system (Section II-B).
* Kinematic trees (``fd_tree``, ``rnea_tree``): ``dense.py``'s definitions with
  Gamma over a parent array.

Parity status: every function is pinned by the CPU tests (closed forms, the
dense definitions, energy and power balance, agreement of independent routes);
none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fd_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

ALGO_CHOLESKY = 0
ALGO_ABA = 1
ALGO_CFA = 2
ALGOS = {"cholesky": ALGO_CHOLESKY, "jsiia": ALGO_CHOLESKY, "aba": ALGO_ABA,
         "abia": ALGO_ABA, "cfa": ALGO_CFA}


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (portable flags, OpenMP across problems)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-Wall",
           "-Wno-unused-function", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            lib = ctypes.CDLL(path)
            dp = ctypes.POINTER(ctypes.c_double)
            i64p = ctypes.POINTER(ctypes.c_int64)
            i32p = ctypes.POINTER(ctypes.c_int32)
            ci = ctypes.c_int
            lib.orc_rnea.argtypes = [ci, dp, dp, dp, dp, dp, dp, dp, dp]
            lib.orc_mass_matrix.argtypes = [ci, dp, dp, dp, dp, dp]
            lib.orc_cfa_blocks.argtypes = [ci, dp, dp, dp, dp, dp, dp, dp, dp, dp, dp, dp]
            lib.orc_oee_solve.argtypes = [ci, ci, dp, dp, dp, dp]
            lib.orc_fd_cfa_w.argtypes = [ci, dp, dp, dp, dp, dp, dp, dp, dp, dp, dp]
            lib.orc_fd_batch.argtypes = [ci, ci, i32p, i64p, i64p, dp, dp, dp, dp, dp, dp,
                                         dp, dp, i32p, ci]
            lib.orc_rnea_batch.argtypes = [ci, i32p, i64p, i64p, dp, dp, dp, dp, dp, dp,
                                           dp, dp, ci]
            for f in (lib.orc_rnea, lib.orc_mass_matrix, lib.orc_cfa_blocks, lib.orc_fd_cfa_w,
                      lib.orc_oee_solve, lib.orc_fd_batch, lib.orc_rnea_batch):
                f.restype = ci
            _lib = lib
    return _lib


def _d(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _chain_arrays(model):
    return _c64(model.axes), _c64(model.frames), _c64(model.inertias), _c64(model.gravity)


def rnea(model, q, qd=None, qdd=None, gravity=None):
    """tau = ID(q, qd, qdd) for a single chain (Eq. 2a-2d)."""
    lib = _load()
    ax, fr, J, g = _chain_arrays(model)
    if gravity is not None:
        g = _c64(gravity)
    n = ax.shape[0]
    tau = np.empty(n)
    q = _c64(q)
    qd = None if qd is None else _c64(qd)
    qdd = None if qdd is None else _c64(qdd)
    st = lib.orc_rnea(n, _d(ax), _d(fr), _d(J), _d(g), _d(q), _d(qd), _d(qdd), _d(tau))
    if st:
        raise RuntimeError(f"oracle rnea failed ({st})")
    return tau


def mass_matrix(model, q):
    """M(q) of a single chain by JSIIA columns (Section II-C)."""
    lib = _load()
    ax, fr, J, _ = _chain_arrays(model)
    n = ax.shape[0]
    M = np.empty((n, n))
    q = _c64(q)
    st = lib.orc_mass_matrix(n, _d(ax), _d(fr), _d(J), _d(q), _d(M))
    if st:
        raise RuntimeError(f"oracle mass matrix failed ({st})")
    return M


def cfa_blocks(model, q, W=None):
    """A (D, U blocks), B (3 blocks per row), C (diagonal, off-diagonal) and W of
    Eq. cfa-eq2 / Eq. fijany-final for a single chain."""
    lib = _load()
    ax, fr, J, _ = _chain_arrays(model)
    n = ax.shape[0]
    D = np.empty((n, 5, 5)); U = np.empty((n, 5, 5)); Bb = np.empty((n, 3, 5))
    Cd = np.empty(n); Co = np.empty(n); Wout = np.empty((n, 6, 5))
    Win = None if W is None else _c64(W)
    q = _c64(q)
    st = lib.orc_cfa_blocks(n, _d(ax), _d(fr), _d(J), _d(q), _d(Win), _d(D), _d(U),
                            _d(Bb), _d(Cd), _d(Co), _d(Wout))
    if st:
        raise RuntimeError(f"oracle cfa blocks failed ({st})")
    return dict(D=D, U=U, B=Bb, Cd=Cd, Co=Co, W=Wout)


def fd_tree(model, q, qd, tau):
    """Forward dynamics of every kinematic tree of a packed model
    (``model.parents``; tree p = problem p) from the dense definitions of
    ``dense`` (Eq. 2a-2d and Eq. 3 with Gamma over the parent array, Eq. 4)."""
    from . import dense
    q, qd, tau = _c64(q), _c64(qd), _c64(tau)
    out = np.full(q.shape[0], np.nan)
    for p in range(model.n_chains):
        a, z = int(model.offsets[p]), int(model.offsets[p + 1])
        if z > a:
            out[a:z] = dense.forward_dynamics(model.chain(p), q[a:z], qd[a:z], tau[a:z])
    return out


def fd_looped(model, q, qd, tau, loops):
    """Forward dynamics of kinematic trees closed by revolute loop joints
    (``loops`` as ``synth.random_loops`` returns; tree p = problem p): the KKT
    system of ``dense.forward_dynamics_looped`` per tree."""
    from . import dense
    q, qd, tau = _c64(q), _c64(qd), _c64(tau)
    out = np.full(q.shape[0], np.nan)
    for p in range(model.n_chains):
        a, z = int(model.offsets[p]), int(model.offsets[p + 1])
        if z == a:
            continue
        sel = np.nonzero(np.asarray(loops["tree"]) == p)[0]
        lp = {k: np.asarray(loops[k])[sel] for k in ("a", "b", "frame_a", "frame_b")}
        out[a:z] = dense.forward_dynamics_looped(model.chain(p), q[a:z], qd[a:z], tau[a:z], lp)
    return out


def rnea_tree(model, q, qd, qdd):
    """Inverse dynamics (with gravity) of every kinematic tree of a packed model
    from the dense Eq. 2a-2d over the parent array."""
    from . import dense
    q, qd, qdd = _c64(q), _c64(qd), _c64(qdd)
    out = np.full(q.shape[0], np.nan)
    for p in range(model.n_chains):
        a, z = int(model.offsets[p]), int(model.offsets[p + 1])
        if z > a:
            out[a:z] = dense.inverse_dynamics(model.chain(p), q[a:z], qd[a:z], qdd[a:z])
    return out


def fd_cfa_w(model, q, qd, tau, W=None, return_fc=False):
    """CFA (Algorithms 1 and 2) with the projection W_i of Eq. cfa-eq1 given per
    link (``W``: L x 6 x 5 in the link frames, W_i^T S_i = 0; None: the default
    complement), chain p = problem p of a packed model. With ``return_fc`` also
    the constraint-force coordinates F_c (L x 5), which depend on W."""
    lib = _load()
    ax, fr, J, g = _chain_arrays(model)
    q, qd, tau = _c64(q), _c64(qd), _c64(tau)
    Wa = None if W is None else _c64(W).reshape(-1, 6, 5)
    L = ax.shape[0]
    qdd = np.full(L, np.nan)
    Fc = np.full((L, 5), np.nan)
    off = np.asarray(model.offsets, dtype=np.int64)
    for p in range(len(off) - 1):
        a, z = int(off[p]), int(off[p + 1])
        if z == a:
            continue
        Wp = None if Wa is None else np.ascontiguousarray(Wa[a:z])
        out = np.empty(z - a)
        fc = np.empty((z - a, 5))
        st = lib.orc_fd_cfa_w(z - a, _d(np.ascontiguousarray(ax[a:z])),
                              _d(np.ascontiguousarray(fr[a:z])),
                              _d(np.ascontiguousarray(J[a:z])), _d(g), _d(q[a:z].copy()),
                              _d(qd[a:z].copy()), _d(tau[a:z].copy()), _d(Wp), _d(out), _d(fc))
        if st:
            raise RuntimeError(f"oracle CFA with a given W failed for chain {p} ({st})")
        qdd[a:z] = out
        Fc[a:z] = fc
    return (qdd, Fc) if return_fc else qdd


def oee_solve(D, U, R):
    """Algorithm 2 on a symmetric block tri-diagonal system. Returns (F, D, U, R)
    after the last level."""
    lib = _load()
    D = _c64(D).copy(); U = _c64(U).copy(); R = _c64(R).copy()
    n, b = R.shape
    F = np.empty((n, b))
    st = lib.orc_oee_solve(n, b, _d(D), _d(U), _d(R), _d(F))
    if st:
        raise RuntimeError(f"oracle OEE failed ({st})")
    return F, D, U, R


def _batch_args(model, chain_index, state_offsets, n_problems):
    if chain_index is None:
        ci = None
        so = np.ascontiguousarray(model.offsets, dtype=np.int64)
    else:
        ci = np.ascontiguousarray(chain_index, dtype=np.int32)
        so = np.ascontiguousarray(state_offsets, dtype=np.int64)
    mo = np.ascontiguousarray(model.offsets, dtype=np.int64)
    return ci, mo, so


def fd(model, q, qd, tau, algo="cholesky", chain_index=None, state_offsets=None,
       n_threads=None, problems=None):
    """Batched forward dynamics qdd = FD(q, qd, tau). ``problems`` optionally
    restricts the computation to a subset of problem indices (others are NaN)."""
    lib = _load()
    ax, fr, J, g = _chain_arrays(model)
    n_problems = model.n_chains if chain_index is None else len(chain_index)
    ci, mo, so = _batch_args(model, chain_index, state_offsets, n_problems)
    q, qd, tau = _c64(q), _c64(qd), _c64(tau)
    qdd = np.full(q.shape[0], np.nan)
    nt = n_threads or 1
    i32p = ctypes.POINTER(ctypes.c_int32)
    i64p = ctypes.POINTER(ctypes.c_int64)
    if problems is not None:
        # one problem per call, so that every problem keeps its batch offsets
        problems = np.asarray(problems, dtype=np.int64)
        status = np.zeros(len(problems), dtype=np.int32)
        for k, p in enumerate(problems):
            so_one = np.array([so[p], so[p + 1]], dtype=np.int64)
            ci_one = np.array([p if ci is None else ci[p]], dtype=np.int32)
            st1 = np.zeros(1, dtype=np.int32)
            lib.orc_fd_batch(ALGOS[algo], 1, ci_one.ctypes.data_as(i32p),
                             mo.ctypes.data_as(i64p), so_one.ctypes.data_as(i64p),
                             _d(ax), _d(fr), _d(J), _d(g), _d(q), _d(qd), _d(tau), _d(qdd),
                             st1.ctypes.data_as(i32p), 1)
            status[k] = st1[0]
    else:
        status = np.zeros(n_problems, dtype=np.int32)
        lib.orc_fd_batch(ALGOS[algo], n_problems,
                         None if ci is None else ci.ctypes.data_as(i32p),
                         mo.ctypes.data_as(i64p), so.ctypes.data_as(i64p),
                         _d(ax), _d(fr), _d(J), _d(g), _d(q), _d(qd), _d(tau), _d(qdd),
                         status.ctypes.data_as(i32p), nt)
    if np.any(status != 0):
        bad = np.nonzero(status)[0]
        raise RuntimeError(f"oracle FD failed for problems {bad[:8]} (status {status[bad[0]]})")
    return qdd


def rnea_batch(model, q, qd, qdd=None, chain_index=None, state_offsets=None, n_threads=None):
    """Batched inverse dynamics tau = ID(q, qd, qdd) with gravity (Eq. 2a-2d)."""
    lib = _load()
    ax, fr, J, g = _chain_arrays(model)
    n_problems = model.n_chains if chain_index is None else len(chain_index)
    ci, mo, so = _batch_args(model, chain_index, state_offsets, n_problems)
    q, qd = _c64(q), _c64(qd)
    qdd = None if qdd is None else _c64(qdd)
    tau = np.empty(q.shape[0])
    i32p = ctypes.POINTER(ctypes.c_int32)
    i64p = ctypes.POINTER(ctypes.c_int64)
    lib.orc_rnea_batch(n_problems, None if ci is None else ci.ctypes.data_as(i32p),
                       mo.ctypes.data_as(i64p), so.ctypes.data_as(i64p), _d(ax), _d(fr),
                       _d(J), _d(g), _d(q), _d(qd), _d(qdd), _d(tau), n_threads or 1)
    return tau
