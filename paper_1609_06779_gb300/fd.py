"""Python binding of the C ABI in include/fd_gb300.h (argument marshalling only).

Every step of forward and inverse dynamics runs in the CUDA library
``libfd_gb300.so``; this module passes torch device pointers and the current
CUDA stream through ctypes. There is no CPU fallback: a missing library or a CPU
tensor raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

ALGOS = {"abia": 0, "jsiia": 1, "cfa": 2, "cfa_cr": 3, "cfa_hybrid": 4, "abia_scan": 5}
PRECS = {"fp64": 0, "fp32": 1, "mixed": 2}
STATUS = {0: "FD_OK", 1: "FD_ERR_INVALID_ARG", 2: "FD_ERR_NOT_SPD", 3: "FD_ERR_OOM",
          4: "FD_ERR_CUDA", 5: "FD_ERR_TIMEOUT", 6: "FD_ERR_NUMERIC", 7: "FD_ERR_BUSY",
          8: "FD_ERR_UNSUPPORTED"}

_lock = threading.Lock()
_lib = None


class FDError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libfd_gb300.so (building it with nvcc if it is missing)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise FDError(4, f"CUDA library not built: {path}")
            _build.build()
        lib = ctypes.CDLL(path)
        vp, sz = ctypes.c_void_p, ctypes.c_size_t
        i32, i64 = ctypes.c_int32, ctypes.c_int64
        dp = ctypes.POINTER(ctypes.c_double)
        i64p = ctypes.POINTER(ctypes.c_int64)
        i32p = ctypes.POINTER(ctypes.c_int32)
        lib.fd_last_error.restype = ctypes.c_char_p
        lib.fd_abi_version.restype = i32
        lib.fd_create_chain.argtypes = [i32, i64p, dp, dp, dp, dp, i32, ctypes.POINTER(vp)]
        lib.fd_create_tree.argtypes = [i32, i64p, i32p, dp, dp, dp, dp, i32,
                                       ctypes.POINTER(vp)]
        lib.fd_tree_add_loops.argtypes = [vp, i32, i32p, i32p, i32p, dp, dp]
        lib.fd_destroy_chain.argtypes = [vp]
        lib.fd_chain_info.argtypes = [vp, i32p, i64p, i32p]
        lib.fd_batch_create.argtypes = [vp, i32, i32p, ctypes.POINTER(vp)]
        lib.fd_batch_destroy.argtypes = [vp]
        lib.fd_batch_info.argtypes = [vp, i32p, i64p, i32p]
        lib.fd_workspace_size.argtypes = [vp, i32, i32, i32]
        lib.fd_workspace_size.restype = sz
        lib.fd_solve_batch.argtypes = [vp, vp, vp, vp, vp, i32, i32, i32, vp, sz, vp, vp]
        lib.fd_inverse_dynamics.argtypes = [vp, vp, vp, vp, vp, i32, i32, vp, sz, vp]
        lib.fd_solve_cfa_static.argtypes = [vp, vp, vp, vp, vp, i32, i32, vp, vp]
        lib.fd_projection_to_canonical.argtypes = [i64, dp, dp, dp]
        lib.fd_solve_cfa_projected.argtypes = [vp, vp, vp, vp, vp, i32, i32, i32, vp, vp, sz,
                                               vp, vp]
        lib.fd_adjoint_workspace_size.argtypes = [vp, i32, i32, i32]
        lib.fd_adjoint_workspace_size.restype = sz
        lib.fd_solve_adjoint.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, i32, i32, i32,
                                         vp, sz, vp, vp]
        lib.fd_solve_adjoint.restype = ctypes.c_int
        lib.fd_autotune.argtypes = [vp, i32, i32, vp, vp, vp, vp, vp, sz, vp,
                                    ctypes.POINTER(i32)]
        lib.fd_autotune.restype = ctypes.c_int
        lib.fd_batch_classes.argtypes = [vp, i32, i32, i32, i32p, i32p, i32p, i32p, i32p]
        lib.fd_measure_fp64_peak.argtypes = [i32, i32, dp, dp]
        lib.fd_measure_fp64_peak.restype = ctypes.c_int
        lib.fd_autotune_cache_load.argtypes = [ctypes.c_char_p, i32p]
        lib.fd_autotune_cache_save.argtypes = [ctypes.c_char_p]
        lib.fd_autotune_cache_clear.argtypes = []
        for f in ("fd_create_chain", "fd_create_tree", "fd_tree_add_loops", "fd_destroy_chain", "fd_chain_info", "fd_batch_create",
                  "fd_batch_destroy", "fd_batch_info", "fd_solve_batch", "fd_inverse_dynamics",
                  "fd_solve_cfa_static", "fd_projection_to_canonical",
                  "fd_solve_cfa_projected", "fd_batch_classes", "fd_autotune_cache_load",
                  "fd_autotune_cache_save", "fd_autotune_cache_clear"):
            getattr(lib, f).restype = ctypes.c_int
        _lib = lib
        return lib


def _check(st: int):
    if st != 0:
        raise FDError(st, load().fd_last_error().decode())


def _dptr(a: np.ndarray):
    return np.ascontiguousarray(a, dtype=np.float64).ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class ChainSet:
    """A set of serial chains resident on one GPU (fd_create_chain), or of
    kinematic trees when ``model.parents`` is set (fd_create_tree: each link's
    parent within its tree, -1 for the base)."""

    def __init__(self, model, device: int = 0):
        lib = load()
        self._lib = lib
        off = np.ascontiguousarray(model.offsets, dtype=np.int64)
        ax = np.ascontiguousarray(model.axes, dtype=np.float64)
        fr = np.ascontiguousarray(model.frames, dtype=np.float64)
        J = np.ascontiguousarray(model.inertias, dtype=np.float64)
        g = np.ascontiguousarray(model.gravity, dtype=np.float64)
        h = ctypes.c_void_p()
        parents = getattr(model, "parents", None)
        if parents is None:
            _check(lib.fd_create_chain(int(off.shape[0] - 1),
                                       off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                       _dptr(ax), _dptr(fr), _dptr(J), _dptr(g), int(device),
                                       ctypes.byref(h)))
        else:
            par = np.ascontiguousarray(parents, dtype=np.int32)
            if par.shape != (int(off[-1]),):
                raise FDError(1, f"parents: need {int(off[-1])} entries, got {par.shape}")
            _check(lib.fd_create_tree(int(off.shape[0] - 1),
                                      off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                      par.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                      _dptr(ax), _dptr(fr), _dptr(J), _dptr(g), int(device),
                                      ctypes.byref(h)))
        self.is_tree = parents is not None
        self.handle = h
        self.device = device
        self.offsets = off.copy()

    def add_loops(self, loops):
        """Close the trees by revolute loop joints (fd_tree_add_loops): ``loops``
        holds arrays tree, a, b (links within the tree, a = -1: the base) and
        frame_a, frame_b (K x 12), as ``synth.random_loops`` returns."""
        i32p = ctypes.POINTER(ctypes.c_int32)
        arr = {k: np.ascontiguousarray(loops[k], dtype=np.int32) for k in ("tree", "a", "b")}
        fa = np.ascontiguousarray(loops["frame_a"], dtype=np.float64).reshape(-1, 12)
        fb = np.ascontiguousarray(loops["frame_b"], dtype=np.float64).reshape(-1, 12)
        K = arr["a"].shape[0]
        _check(self._lib.fd_tree_add_loops(self.handle, K, arr["tree"].ctypes.data_as(i32p),
                                           arr["a"].ctypes.data_as(i32p),
                                           arr["b"].ctypes.data_as(i32p), _dptr(fa), _dptr(fb)))

    def info(self):
        n = ctypes.c_int32(); L = ctypes.c_int64(); m = ctypes.c_int32()
        _check(self._lib.fd_chain_info(self.handle, ctypes.byref(n), ctypes.byref(L),
                                       ctypes.byref(m)))
        return n.value, L.value, m.value

    def close(self):
        if getattr(self, "handle", None):
            self._lib.fd_destroy_chain(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """A batch plan (fd_batch_create): problem p uses chain chain_index[p]."""

    def __init__(self, chains: ChainSet, chain_index=None):
        lib = load()
        self._lib = lib
        self.chains = chains
        h = ctypes.c_void_p()
        if chain_index is None:
            n_problems = chains.info()[0]
            _check(lib.fd_batch_create(chains.handle, n_problems, None, ctypes.byref(h)))
        else:
            ci = np.ascontiguousarray(chain_index, dtype=np.int32)
            n_problems = int(ci.shape[0])
            _check(lib.fd_batch_create(chains.handle, n_problems,
                                       ci.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                       ctypes.byref(h)))
        self.handle = h
        n = ctypes.c_int32(); L = ctypes.c_int64(); m = ctypes.c_int32()
        _check(lib.fd_batch_info(h, ctypes.byref(n), ctypes.byref(L), ctypes.byref(m)))
        self.n_problems, self.n_state_links, self.max_links = n.value, L.value, m.value

    def workspace_size(self, algo, prec="fp64", team=0) -> int:
        a = -1 if algo in (None, "id") else ALGOS[algo]
        return int(self._lib.fd_workspace_size(self.handle, a, PRECS[prec], int(team)))

    def close(self):
        if getattr(self, "handle", None):
            self._lib.fd_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _torch():
    import torch
    return torch


def _state_dtype(prec):
    torch = _torch()
    return torch.float64 if prec == "fp64" else torch.float32


def _check_state(t, batch, dtype, name):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise FDError(1, f"{name} must be a CUDA tensor (there is no CPU path)")
    if t.dtype != dtype or not t.is_contiguous() or t.numel() != batch.n_state_links:
        raise FDError(1, f"{name}: need contiguous {dtype} of {batch.n_state_links} elements, "
                         f"got {t.dtype} {tuple(t.shape)}")


def workspace(batch: Batch, algo, prec="fp64", team=0, device=None):
    torch = _torch()
    n = batch.workspace_size(algo, prec, team)
    # the caching allocator returns blocks aligned to at least 512 bytes
    return torch.empty(max(n, 1), dtype=torch.uint8,
                       device=device if device is not None else f"cuda:{batch.chains.device}")


def solve(batch: Batch, q, qd, tau, algo="cfa", prec="fp64", team=0, out=None, ws=None,
          status=None, stream=None):
    """qdd = FD(q, qd, tau) for every problem of ``batch`` (fd_solve_batch)."""
    torch = _torch()
    dt = _state_dtype(prec)
    for t, nm in ((q, "q"), (qd, "qdot"), (tau, "tau")):
        _check_state(t, batch, dt, nm)
    if out is None:
        out = torch.empty_like(q)
    _check_state(out, batch, dt, "qddot")
    if ws is None:
        ws = workspace(batch, algo, prec, team, q.device)
    if status is not None and (status.dtype != torch.int32 or not status.is_cuda
                               or status.numel() < batch.n_problems):
        raise FDError(1, "status must be a CUDA int32 tensor of n_problems elements")
    s = stream if stream is not None else torch.cuda.current_stream(q.device)
    _check(load().fd_solve_batch(batch.handle, q.data_ptr(), qd.data_ptr(), tau.data_ptr(),
                                 out.data_ptr(), ALGOS[algo], PRECS[prec], int(team),
                                 ws.data_ptr(), ws.numel(),
                                 None if status is None else status.data_ptr(),
                                 ctypes.c_void_p(s.cuda_stream)))
    return out


def inverse_dynamics(batch: Batch, q, qd, qdd, prec="fp64", team=0, out=None, ws=None,
                     stream=None):
    """tau = ID(q, qd, qdd) with gravity (fd_inverse_dynamics)."""
    torch = _torch()
    dt = _state_dtype(prec)
    for t, nm in ((q, "q"), (qd, "qdot"), (qdd, "qddot")):
        _check_state(t, batch, dt, nm)
    if out is None:
        out = torch.empty_like(q)
    if ws is None:
        ws = workspace(batch, None, prec, team, q.device)
    s = stream if stream is not None else torch.cuda.current_stream(q.device)
    _check(load().fd_inverse_dynamics(batch.handle, q.data_ptr(), qd.data_ptr(), qdd.data_ptr(),
                                      out.data_ptr(), PRECS[prec], int(team), ws.data_ptr(),
                                      ws.numel(), ctypes.c_void_p(s.cuda_stream)))
    return out


PROJECTIONS = {"canonical": 0, "given": 1, "block_jacobi": 2}


def projection_to_canonical(joint_axes, W) -> np.ndarray:
    """Q_i (n x 5 x 5) of projections W_i (n x 6 x 5, link frames, (omega; v)
    order; fd_projection_to_canonical): W_i = Wc_i Q_i, Wc_i the library's own
    complement of the joint axis. Host only."""
    ax = np.ascontiguousarray(joint_axes, dtype=np.float64).reshape(-1, 3)
    Wa = np.ascontiguousarray(W, dtype=np.float64).reshape(ax.shape[0], 6, 5)
    Q = np.empty((ax.shape[0], 5, 5))
    _check(load().fd_projection_to_canonical(ax.shape[0], _dptr(ax), _dptr(Wa), _dptr(Q)))
    return Q


def solve_cfa_projected(batch: Batch, q, qd, tau, projection="block_jacobi", Q=None,
                        prec="fp64", team=0, out=None, ws=None, status=None, stream=None):
    """CFA on the system of a general projection W_i = Wc_i Q_i
    (fd_solve_cfa_projected): ``projection`` is "canonical", "given" (``Q``: a
    CUDA float64 tensor of the chain set's n_links x 5 x 5 entries, from
    :func:`projection_to_canonical`) or "block_jacobi". FP64 or FP32."""
    torch = _torch()
    dt = _state_dtype(prec)
    for t, nm in ((q, "q"), (qd, "qdot"), (tau, "tau")):
        _check_state(t, batch, dt, nm)
    if out is None:
        out = torch.empty_like(q)
    _check_state(out, batch, dt, "qddot")
    if projection not in PROJECTIONS:
        raise FDError(1, f"unknown projection {projection!r}")
    qptr = None
    if projection == "given":
        n_links = batch.chains.info()[1]
        if (not isinstance(Q, torch.Tensor) or not Q.is_cuda or Q.dtype != torch.float64
                or not Q.is_contiguous() or Q.numel() != 25 * n_links):
            raise FDError(1, f"Q must be a contiguous CUDA float64 tensor of {25 * n_links} "
                             f"entries")
        qptr = Q.data_ptr()
    if ws is None:
        ws = workspace(batch, "cfa", prec, team, q.device)
    if status is not None and (status.dtype != torch.int32 or not status.is_cuda
                               or status.numel() < batch.n_problems):
        raise FDError(1, "status must be a CUDA int32 tensor of n_problems elements")
    s = stream if stream is not None else torch.cuda.current_stream(q.device)
    _check(load().fd_solve_cfa_projected(batch.handle, q.data_ptr(), qd.data_ptr(),
                                         tau.data_ptr(), out.data_ptr(), PRECS[prec], int(team),
                                         PROJECTIONS[projection], qptr, ws.data_ptr(),
                                         ws.numel(),
                                         None if status is None else status.data_ptr(),
                                         ctypes.c_void_p(s.cuda_stream)))
    return out


def solve_cfa_static(chains: ChainSet, q, qd, tau, prec="fp64", team=0, out=None, status=None,
                     stream=None):
    """CFA for problem p = chain p with the library's static scratch
    (fd_solve_cfa_static): no allocation by the library; ``out`` may be given to
    avoid torch's allocation as well."""
    torch = _torch()
    dt = _state_dtype(prec)
    n_chains, n_links = chains.info()[0], chains.info()[1]

    def check(t, nm):
        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != dt \
                or not t.is_contiguous() or t.numel() != n_links:
            raise FDError(1, f"{nm}: need a contiguous CUDA {dt} tensor of {n_links} elements")
    for t, nm in ((q, "q"), (qd, "qdot"), (tau, "tau")):
        check(t, nm)
    if out is None:
        out = torch.empty_like(q)
    check(out, "qddot")
    if status is not None and (not isinstance(status, torch.Tensor) or not status.is_cuda
                               or status.dtype != torch.int32 or not status.is_contiguous()
                               or status.numel() < n_chains):
        raise FDError(1, f"status must be a contiguous CUDA int32 tensor of at least "
                         f"{n_chains} elements")
    s = stream if stream is not None else torch.cuda.current_stream(q.device)
    _check(load().fd_solve_cfa_static(chains.handle, q.data_ptr(), qd.data_ptr(), tau.data_ptr(),
                                      out.data_ptr(), PRECS[prec], int(team),
                                      None if status is None else status.data_ptr(),
                                      ctypes.c_void_p(s.cuda_stream)))
    return out


def adjoint(batch: Batch, q, qd, tau, qdd_bar, qdd=None, algo="cfa", prec="fp64", team=0,
            masses=True, ws=None, status=None, stream=None):
    """Reverse-mode derivatives of qdd = FD(q, qd, tau) for the cotangent
    ``qdd_bar`` (fd_solve_adjoint). Returns (q_bar, qd_bar, tau_bar, mass_bar);
    mass_bar is None unless ``masses``."""
    torch = _torch()
    dt = _state_dtype(prec)
    for t, nm in ((q, "q"), (qd, "qdot"), (tau, "tau"), (qdd_bar, "qddot_bar")):
        _check_state(t, batch, dt, nm)
    if qdd is not None:
        _check_state(qdd, batch, dt, "qddot")
    outs = [torch.empty_like(q) for _ in range(4 if masses else 3)]
    if ws is None:
        n = int(load().fd_adjoint_workspace_size(batch.handle, ALGOS[algo], PRECS[prec],
                                                 int(team)))
        ws = torch.empty(max(n, 1), dtype=torch.uint8, device=q.device)
    s = stream if stream is not None else torch.cuda.current_stream(q.device)
    _check(load().fd_solve_adjoint(batch.handle, q.data_ptr(), qd.data_ptr(), tau.data_ptr(),
                                   None if qdd is None else qdd.data_ptr(), qdd_bar.data_ptr(),
                                   outs[0].data_ptr(), outs[1].data_ptr(), outs[2].data_ptr(),
                                   outs[3].data_ptr() if masses else None, ALGOS[algo],
                                   PRECS[prec], int(team), ws.data_ptr(), ws.numel(),
                                   None if status is None else status.data_ptr(),
                                   ctypes.c_void_p(s.cuda_stream)))
    return outs[0], outs[1], outs[2], (outs[3] if masses else None)


def _make_autograd():
    torch = _torch()

    class ForwardDynamics(torch.autograd.Function):
        """qdd = FD(q, qd, tau) with the adjoint kernels as its backward."""

        @staticmethod
        def forward(ctx, q, qd, tau, batch, algo, prec, team):
            qdd = solve(batch, q.contiguous(), qd.contiguous(), tau.contiguous(), algo=algo,
                        prec=prec, team=team)
            ctx.save_for_backward(q, qd, tau, qdd)
            ctx.cfg = (batch, algo, prec, team)
            return qdd

        @staticmethod
        def backward(ctx, g):
            q, qd, tau, qdd = ctx.saved_tensors
            batch, algo, prec, team = ctx.cfg
            qb, qdb, tb, _ = adjoint(batch, q, qd, tau, g.contiguous(), qdd=qdd, algo=algo,
                                     prec=prec, team=team, masses=False)
            return qb, qdb, tb, None, None, None, None

    return ForwardDynamics


_FD_FN = None


def forward_dynamics(batch: Batch, q, qd, tau, algo="cfa", prec="fp64", team=0):
    """Differentiable qdd = FD(q, qd, tau) (torch.autograd.Function)."""
    global _FD_FN
    if _FD_FN is None:
        _FD_FN = _make_autograd()
    return _FD_FN.apply(q, qd, tau, batch, algo, prec, team)


def autotune(batch: Batch, q, qd, tau, algo="cfa", prec="fp64", max_workspace_bytes=32 << 30,
             stream=None) -> int:
    """Time the team sizes (fd_autotune) and record the fastest in the batch plan;
    returns it, or 0 for a batch of several length classes (then every class has
    its own team: see :func:`batch_classes`). Team sizes whose workspace exceeds
    ``max_workspace_bytes`` are skipped, except the smallest. Entries of the
    process-wide autotune cache (:func:`autotune_cache_load`) are used without
    timing."""
    torch = _torch()
    dt = _state_dtype(prec)
    for t, nm in ((q, "q"), (qd, "qdot"), (tau, "tau")):
        _check_state(t, batch, dt, nm)
    need = batch.workspace_size(algo, prec, 1)
    t = 2
    while t <= 256:
        n = batch.workspace_size(algo, prec, t)
        if n <= max_workspace_bytes:
            need = max(need, n)
        t *= 2
    ws = torch.empty(max(need, 1), dtype=torch.uint8, device=q.device)
    out = torch.empty_like(q)
    best = ctypes.c_int32(0)
    s = stream if stream is not None else torch.cuda.current_stream(q.device)
    _check(load().fd_autotune(batch.handle, ALGOS[algo], PRECS[prec], q.data_ptr(), qd.data_ptr(),
                              tau.data_ptr(), out.data_ptr(), ws.data_ptr(), ws.numel(),
                              ctypes.c_void_p(s.cuda_stream), ctypes.byref(best)))
    return best.value


def batch_classes(batch: Batch, algo="cfa", prec="fp64"):
    """The batch's length classes (fd_batch_classes): a list of dicts with the
    class's shortest and longest chain, its problem count and the team a team-0
    solve of ``algo`` / ``prec`` runs it with."""
    lib = load()
    n = ctypes.c_int32(0)
    _check(lib.fd_batch_classes(batch.handle, ALGOS[algo] if algo else -1, PRECS[prec], 0,
                                ctypes.byref(n), None, None, None, None))
    k = n.value
    arrs = [(ctypes.c_int32 * max(k, 1))() for _ in range(4)]
    _check(lib.fd_batch_classes(batch.handle, ALGOS[algo] if algo else -1, PRECS[prec], k,
                                ctypes.byref(n), *arrs))
    return [{"min_len": arrs[0][c], "max_len": arrs[1][c], "count": arrs[2][c],
             "team": arrs[3][c]} for c in range(k)]


def measure_fp64_peak(device=0, iters=200000):
    """FP64 TFLOP/s of independent fused multiply-adds on this GPU and the timed
    kernel's milliseconds (fd_measure_fp64_peak)."""
    tf, ms = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(load().fd_measure_fp64_peak(int(device), int(iters), ctypes.byref(tf),
                                       ctypes.byref(ms)))
    return tf.value, ms.value


def autotune_cache_load(path) -> int:
    """Merge a saved autotune cache into the process-wide one (a missing file
    loads nothing); returns the number of entries read."""
    n = ctypes.c_int32(0)
    _check(load().fd_autotune_cache_load(os.fsencode(path), ctypes.byref(n)))
    return n.value


def autotune_cache_save(path):
    """Write the process-wide autotune cache as JSON."""
    _check(load().fd_autotune_cache_save(os.fsencode(path)))


def autotune_cache_clear():
    _check(load().fd_autotune_cache_clear())


# ------------------------------------------------------------------- serving

class _Request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("algo", ctypes.c_int32), ("model_id", ctypes.c_int32),
                ("steps", ctypes.c_int32), ("dt", ctypes.c_double),
                ("q", ctypes.c_void_p), ("qdot", ctypes.c_void_p), ("tau", ctypes.c_void_p),
                ("qddot_bar", ctypes.c_void_p)]


class _Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("n_links", ctypes.c_int32),
                ("steps_done", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("submit_time", ctypes.c_double), ("done_time", ctypes.c_double),
                ("q", ctypes.c_void_p), ("qdot", ctypes.c_void_p), ("qddot", ctypes.c_void_p),
                ("q_bar", ctypes.c_void_p), ("qdot_bar", ctypes.c_void_p),
                ("tau_bar", ctypes.c_void_p)]


class _Stats(ctypes.Structure):
    _fields_ = [("ticks", ctypes.c_uint64), ("launches", ctypes.c_uint64),
                ("completed", ctypes.c_uint64), ("queued", ctypes.c_uint64),
                ("active", ctypes.c_uint64), ("link_slots_used", ctypes.c_int64),
                ("link_slots", ctypes.c_int64), ("link_solves", ctypes.c_double),
                ("busy_seconds", ctypes.c_double)]


REQ_FD_GRAD, REQ_ROLLOUT = 0, 1
SERVE_PER_SIZE = 1


def _serve_lib():
    lib = load()
    if not getattr(lib, "_serve_ready", False):
        vp, sz = ctypes.c_void_p, ctypes.c_size_t
        i32, u64 = ctypes.c_int32, ctypes.c_uint64
        dp = ctypes.POINTER(ctypes.c_double)
        lib.fd_serve_clock.restype = ctypes.c_double
        lib.fd_serve_create.argtypes = [i32, sz, dp, i32, ctypes.POINTER(vp)]
        lib.fd_serve_add_model.argtypes = [vp, i32, dp, dp, dp, ctypes.POINTER(i32)]
        lib.fd_serve_remove_model.argtypes = [vp, i32]
        lib.fd_serve_submit.argtypes = [vp, ctypes.POINTER(_Request), ctypes.POINTER(u64)]
        lib.fd_serve_poll.argtypes = [vp, u64, ctypes.POINTER(_Result)]
        lib.fd_serve_wait.argtypes = [vp, u64, i32, ctypes.POINTER(_Result)]
        lib.fd_serve_drain.argtypes = [vp, i32, ctypes.POINTER(u64), dp, dp,
                                       ctypes.POINTER(i32), ctypes.POINTER(i32)]
        lib.fd_serve_stats.argtypes = [vp, ctypes.POINTER(_Stats)]
        lib.fd_serve_destroy.argtypes = [vp]
        for f in ("fd_serve_create", "fd_serve_add_model", "fd_serve_remove_model",
                  "fd_serve_submit", "fd_serve_poll", "fd_serve_wait", "fd_serve_drain",
                  "fd_serve_stats", "fd_serve_destroy"):
            getattr(lib, f).restype = ctypes.c_int
        lib._serve_ready = True
    return lib


def serve_clock() -> float:
    return float(_serve_lib().fd_serve_clock())


class Server:
    """Continuous-batching forward-dynamics server (fd_serve_*)."""

    def __init__(self, device=0, budget_bytes=1 << 30, gravity=(0.0, 0.0, -9.81),
                 per_size=False):
        lib = _serve_lib()
        self._lib = lib
        g = np.ascontiguousarray(gravity, dtype=np.float64)
        h = ctypes.c_void_p()
        _check(lib.fd_serve_create(int(device), int(budget_bytes), _dptr(g),
                                   SERVE_PER_SIZE if per_size else 0, ctypes.byref(h)))
        self.handle = h
        self.n_of = {}

    def add_model(self, model) -> int:
        """Register one chain (a ChainModel with a single chain)."""
        ax = np.ascontiguousarray(model.axes, dtype=np.float64)
        fr = np.ascontiguousarray(model.frames, dtype=np.float64)
        J = np.ascontiguousarray(model.inertias, dtype=np.float64)
        mid = ctypes.c_int32()
        _check(self._lib.fd_serve_add_model(self.handle, ax.shape[0], _dptr(ax), _dptr(fr),
                                            _dptr(J), ctypes.byref(mid)))
        self.n_of[mid.value] = ax.shape[0]
        return mid.value

    def remove_model(self, model_id):
        _check(self._lib.fd_serve_remove_model(self.handle, int(model_id)))

    def _submit(self, kind, algo, model_id, q, qd, tau, w=None, steps=1, dt=0.0):
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (q, qd, tau)]
        wv = None if w is None else np.ascontiguousarray(w, dtype=np.float64)
        rq = _Request(kind, ALGOS[algo], int(model_id), int(steps), float(dt),
                      arrs[0].ctypes.data, arrs[1].ctypes.data, arrs[2].ctypes.data,
                      None if wv is None else wv.ctypes.data)
        t = ctypes.c_uint64()
        _check(self._lib.fd_serve_submit(self.handle, ctypes.byref(rq), ctypes.byref(t)))
        return t.value

    def submit_grad(self, model_id, q, qd, tau, qdd_bar, algo="cfa") -> int:
        return self._submit(REQ_FD_GRAD, algo, model_id, q, qd, tau, qdd_bar)

    def submit_rollout(self, model_id, q, qd, taus, dt, algo="abia") -> int:
        taus = np.ascontiguousarray(taus, dtype=np.float64)
        return self._submit(REQ_ROLLOUT, algo, model_id, q, qd, taus.reshape(-1),
                            steps=taus.shape[0], dt=dt)

    def wait(self, ticket, timeout_ms=60000, n=4096):
        """Blocks up to timeout_ms; returns a dict of results (raises FDError on
        FD_ERR_TIMEOUT and other failures). ``n``: at least the chain's links."""
        bufs = {k: np.full(n, np.nan) for k in ("q", "qdot", "qddot", "q_bar", "qdot_bar",
                                                  "tau_bar")}
        res = _Result()
        for k, v in bufs.items():
            setattr(res, k, v.ctypes.data)
        _check(self._lib.fd_serve_wait(self.handle, int(ticket), int(timeout_ms),
                                       ctypes.byref(res)))
        m = res.n_links
        out = {k: v[:m].copy() for k, v in bufs.items()}
        out.update(status=res.status, steps_done=res.steps_done, submit_time=res.submit_time,
                   done_time=res.done_time)
        return out

    def drain(self, max_n=65536):
        """Finished requests: (tickets, submit times, done times, statuses)."""
        if getattr(self, "_dbuf", None) is None or self._dbuf[0] < max_n:
            self._dbuf = (max_n, (ctypes.c_uint64 * max_n)(), np.empty(max_n), np.empty(max_n),
                          (ctypes.c_int32 * max_n)(), ctypes.c_int32())
        _, t, sub, done, st, cnt = self._dbuf
        _check(self._lib.fd_serve_drain(self.handle, max_n, t, _dptr(sub), _dptr(done), st,
                                        ctypes.byref(cnt)))
        k = cnt.value
        return (np.frombuffer(t, dtype=np.uint64)[:k].copy(), sub[:k].copy(), done[:k].copy(),
                np.frombuffer(st, dtype=np.int32)[:k].copy())

    def stats(self):
        s = _Stats()
        _check(self._lib.fd_serve_stats(self.handle, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in _Stats._fields_}

    def close(self):
        if getattr(self, "handle", None):
            self._lib.fd_serve_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
