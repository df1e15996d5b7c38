"""Stored oracle values (tests/golden/, written by tests/golden/make_golden.py).

The paper prints no worked example, so the stored values are the FP64 oracle's
own results on small seeded chains. CPU: the oracle still reproduces them (a
change to its arithmetic shows up here) and its three routes agree on them.
GPU: the CUDA path meets them through the C ABI without running the oracle."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1609_06779_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden")
FILES = sorted(f for f in os.listdir(GOLDEN) if f.endswith(".json"))


def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        g = json.load(f)
    model = synth.random_chains(g["lengths"], seed=g["model_seed"])
    st = synth.random_states(model.n_links_total, seed=g["state_seed"])
    qdd_in = np.random.default_rng(g["state_seed"] + 1).standard_normal(model.n_links_total)
    return g, model, st, qdd_in


def _rel(got, ref, offsets):
    out = []
    for a, b in zip(offsets[:-1], offsets[1:]):
        out.append(np.abs(got[a:b] - ref[a:b]).max() / max(np.abs(ref[a:b]).max(), 1e-300))
    return np.array(out)


def test_golden_files_present():
    assert FILES, "tests/golden holds no stored values"


@pytest.mark.parametrize("name", FILES)
def test_oracle_reproduces_stored_values(name):
    # not bit for bit: gcc may contract a * b + c differently on another host
    g, model, st, qdd_in = _load(name)
    off = model.offsets
    for algo in ("cholesky", "aba", "cfa"):
        got = oracle.fd(model, st.q, st.qdot, st.tau, algo=algo)
        assert _rel(got, np.array(g[f"qdd_{algo}"]), off).max() < 1e-12, algo
    tau = oracle.rnea_batch(model, st.q, st.qdot, qdd_in)
    assert _rel(tau, np.array(g["tau_id"]), off).max() < 1e-12


@pytest.mark.parametrize("name", FILES)
def test_stored_routes_agree(name):
    g, model, _, _ = _load(name)
    ref = np.array(g["qdd_cholesky"])
    for algo in ("aba", "cfa"):
        assert _rel(np.array(g[f"qdd_{algo}"]), ref, model.offsets).max() < 1e-10, algo


@pytest.mark.gpu
@pytest.mark.parametrize("name", FILES)
def test_cuda_path_meets_stored_values(name):
    torch = pytest.importorskip("torch")
    from paper_1609_06779_gb300 import fd
    g, model, st, qdd_in = _load(name)
    off = model.offsets
    ref = np.array(g["qdd_cholesky"])
    cs = fd.ChainSet(model)
    b = fd.Batch(cs)
    t = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")
    q, qd, tau = t(st.q), t(st.qdot), t(st.tau)
    for algo, team in (("abia", 1), ("abia", 8), ("jsiia", 2), ("jsiia", 8), ("cfa", 8),
                       ("cfa", 32), ("cfa_cr", 8)):
        got = fd.solve(b, q, qd, tau, algo=algo, team=team).cpu().numpy()
        assert _rel(got, ref, off).max() < 1e-10, (algo, team)
    tau_id = fd.inverse_dynamics(b, q, qd, t(qdd_in), team=8).cpu().numpy()
    assert _rel(tau_id, np.array(g["tau_id"]), off).max() < 1e-12
