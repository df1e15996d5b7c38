"""Host-side checks of the C ABI that need no GPU: the library builds, exports
every entry point that include/fd_gb300.h declares, validates its arguments
before touching the device, and fails loudly (no CPU fallback) without one."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1609_06779_gb300 import build as fdbuild
from paper_1609_06779_gb300 import fd, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(fd_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    fdbuild.build()
    return fd.load()


def test_library_exports_every_declared_symbol(lib):
    declared = _declared_functions()
    assert "fd_solve_batch" in declared and "fd_create_chain" in declared
    for name in declared:
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"
    assert lib.fd_abi_version() == 1


def _create(model, lib):
    h = ctypes.c_void_p()
    off = np.ascontiguousarray(model.offsets, dtype=np.int64)
    dp = lambda a: np.ascontiguousarray(a, dtype=np.float64).ctypes.data_as(
        ctypes.POINTER(ctypes.c_double))
    st = lib.fd_create_chain(int(off.shape[0] - 1),
                             off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                             dp(model.axes), dp(model.frames), dp(model.inertias),
                             dp(model.gravity), 0, ctypes.byref(h))
    return st, h


def test_invalid_models_rejected_before_any_device_call(lib):
    base = synth.random_chains([3, 2], seed=0)

    def variant(fn):
        m = synth.random_chains([3, 2], seed=0)
        fn(m)
        return m

    cases = {
        "zero axis": variant(lambda m: m.axes.__setitem__(1, 0.0)),
        "not a rotation": variant(lambda m: m.frames.__setitem__((0, 0), 2.0)),
        "reflection": variant(lambda m: m.frames.__setitem__((0, slice(0, 9)),
                                                             np.diag([1, 1, -1.0]).reshape(9))),
        "non-symmetric inertia": variant(lambda m: m.inertias.__setitem__((2, 1), 5.0)),
        "indefinite inertia": variant(lambda m: m.inertias.__setitem__(
            (4, slice(None)), (-np.eye(6)).reshape(36))),
        "nan gravity": variant(lambda m: m.gravity.__setitem__(0, np.nan)),
    }
    for name, m in cases.items():
        st, h = _create(m, lib)
        assert st == 1, name
        assert h.value is None
        assert len(lib.fd_last_error()) > 0
    bad_off = synth.random_chains([3, 2], seed=0)
    bad_off.offsets = np.array([0, 4, 3], dtype=np.int64)
    assert _create(bad_off, lib)[0] == 1
    # a valid model gets past validation; without a GPU the call must fail loudly
    st, h = _create(base, lib)
    if st != 0:
        assert st == 4, fd.STATUS.get(st)
        assert b"CUDA" in lib.fd_last_error() or b"device" in lib.fd_last_error()
    else:
        lib.fd_destroy_chain(h)


def test_null_handles_are_invalid(lib):
    assert lib.fd_destroy_chain(None) == 1
    assert lib.fd_batch_destroy(None) == 1
    assert lib.fd_solve_batch(None, None, None, None, None, 2, 0, 0, None, 0, None, None) == 1
    assert lib.fd_inverse_dynamics(None, None, None, None, None, 0, 0, None, 0, None) == 1
    assert lib.fd_workspace_size(None, 2, 0, 0) == 0


def test_python_binding_refuses_cpu_tensors():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("checks the no-GPU path")
    with pytest.raises(fd.FDError):
        fd.ChainSet(synth.random_chains([2], seed=0))


def test_server_without_a_device_fails_loudly(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("checks the no-GPU path")
    g = (ctypes.c_double * 3)(0.0, 0.0, -9.81)
    h = ctypes.c_void_p()
    lib.fd_serve_create.argtypes = [ctypes.c_int32, ctypes.c_size_t,
                                    ctypes.POINTER(ctypes.c_double), ctypes.c_int32,
                                    ctypes.POINTER(ctypes.c_void_p)]
    assert lib.fd_serve_create(0, 64 << 20, g, 0, ctypes.byref(h)) == 4
    assert lib.fd_serve_create(0, 1 << 10, g, 0, ctypes.byref(h)) == 1   # budget too small
    assert h.value is None


def test_autotune_cache_round_trip(lib, tmp_path):
    """The autotune cache is host-only JSON: a saved cache loads back, a missing
    file loads nothing, a malformed one is rejected."""
    import json
    fd.autotune_cache_clear()
    assert fd.autotune_cache_load(str(tmp_path / "missing.json")) == 0
    src = {"format": "fd_gb300 autotune cache 1", "entries": [
        {"gpu": "NVIDIA GB300 (152 SMs)", "algo": 2, "prec": 0, "len_class": 5,
         "count_class": 16, "team": 8, "ms": 11.0},
        {"gpu": "NVIDIA GB300 (152 SMs)", "algo": 0, "prec": 2, "len_class": 9,
         "count_class": 10, "team": 32, "ms": 3.2}]}
    p = tmp_path / "cache.json"
    p.write_text(json.dumps(src))
    assert fd.autotune_cache_load(str(p)) == 2
    out = tmp_path / "saved.json"
    fd.autotune_cache_save(str(out))
    got = json.loads(out.read_text())
    assert got["format"] == src["format"]
    key = lambda e: (e["algo"], e["prec"], e["len_class"], e["count_class"], e["team"])
    assert sorted(map(key, got["entries"])) == sorted(map(key, src["entries"]))
    bad = tmp_path / "bad.json"
    bad.write_text(json.dumps({"format": "fd_gb300 autotune cache 1", "entries": [
        {"gpu": "x", "algo": 0, "prec": 0, "len_class": 1, "count_class": 1, "team": 4}]}))
    with pytest.raises(fd.FDError):          # ABIA has no team of 4
        fd.autotune_cache_load(str(bad))
    bad.write_text("{}")
    with pytest.raises(fd.FDError):
        fd.autotune_cache_load(str(bad))
    fd.autotune_cache_clear()
    fd.autotune_cache_save(str(out))
    assert json.loads(out.read_text())["entries"] == []


def test_projection_to_canonical(lib):
    """fd_projection_to_canonical (host only): an orthonormal complement of each
    joint axis maps to an orthogonal Q_i, W_i Z_i maps to Q_i Z_i, and a W_i that
    is not a complement of S_i, or has rank below 5, is rejected."""
    import oracle.dense as dense
    model = synth.random_chains([4, 3], seed=5)
    L = model.n_links_total
    _, Wb = dense.projection(model)
    Q = fd.projection_to_canonical(model.axes, Wb)
    for i in range(L):
        np.testing.assert_allclose(Q[i].T @ Q[i], np.eye(5), atol=1e-13)
    rng = np.random.default_rng(1)
    Z = rng.standard_normal((L, 5, 5)) + 2 * np.eye(5)
    Qz = fd.projection_to_canonical(model.axes, Wb @ Z)
    np.testing.assert_allclose(Qz, Q @ Z, atol=1e-12)
    bad = Wb.copy()
    bad[2, :3, 1] += np.asarray(model.axes)[2] / np.linalg.norm(model.axes[2])  # S^T W != 0
    with pytest.raises(fd.FDError, match="W\\^T S"):
        fd.projection_to_canonical(model.axes, bad)
    low = Wb.copy()
    low[1, :, 4] = low[1, :, 3]  # two equal columns
    with pytest.raises(fd.FDError, match="rank"):
        fd.projection_to_canonical(model.axes, low)
    assert fd.projection_to_canonical(np.zeros((0, 3)), np.zeros((0, 6, 5))).shape == (0, 5, 5)


def test_create_tree_validates_parents_before_any_device_call(lib):
    """fd_create_tree: each link's parent must be -1 or an earlier link of the
    same tree; a NULL parent array with links is rejected."""
    m = synth.random_chains([4, 3], seed=2)
    off = np.ascontiguousarray(m.offsets, dtype=np.int64)
    dp = lambda a: np.ascontiguousarray(a, dtype=np.float64).ctypes.data_as(
        ctypes.POINTER(ctypes.c_double))

    def create(parents):
        h = ctypes.c_void_p()
        par = None if parents is None else np.ascontiguousarray(parents, dtype=np.int32)
        return lib.fd_create_tree(2, off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                  None if par is None else par.ctypes.data_as(
                                      ctypes.POINTER(ctypes.c_int32)),
                                  dp(m.axes), dp(m.frames), dp(m.inertias), dp(m.gravity), 0,
                                  ctypes.byref(h))
    assert create([-1, 0, 1, 3, -1, 0, 0]) == 1      # link 3 is its own parent
    assert create([-1, 0, 1, 1, -1, 0, 5]) == 1      # parent beyond the link
    assert create([-1, 0, -2, 1, -1, 0, 0]) == 1     # parent below -1
    assert create(None) == 1
    assert b"parent" in lib.fd_last_error()
