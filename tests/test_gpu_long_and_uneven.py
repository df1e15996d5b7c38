"""Long chains (256 and 1024 links) and an uneven batch with lengths log-uniform
in [6, 512]: parity with the FP64 oracle on sampled chains, properties on all."""
import numpy as np
import pytest

import oracle
from paper_1609_06779_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

EPS32 = float(np.finfo(np.float32).eps)


def _rel_err(got, ref, offsets):
    errs = []
    for p in range(len(offsets) - 1):
        a, b = offsets[p], offsets[p + 1]
        if b > a:
            errs.append(np.abs(got[a:b] - ref[a:b]).max() / max(np.abs(ref[a:b]).max(), 1e-300))
    return np.array(errs)


def _gpu(model, st, algo, prec, team):
    from paper_1609_06779_gb300 import fd
    cs = fd.ChainSet(model)
    b = fd.Batch(cs)
    dt = torch.float64 if prec == "fp64" else torch.float32
    t = lambda a: torch.tensor(a, dtype=dt, device="cuda")
    status = torch.full((b.n_problems,), -1, dtype=torch.int32, device="cuda")
    out = fd.solve(b, t(st.q), t(st.qdot), t(st.tau), algo=algo, prec=prec, team=team,
                   status=status)
    torch.cuda.synchronize()
    return out.double().cpu().numpy(), status.cpu().numpy()


@pytest.mark.parametrize("n,count", [(256, 6), (1024, 3)])
def test_long_chains_fp64(n, count):
    model = synth.random_chains([n] * count, seed=n)
    st = synth.random_states(model.n_links_total, seed=n + 1)
    ref = oracle.fd(model, st.q, st.qdot, st.tau, algo="cholesky", n_threads=8)
    # the error floor of each algorithm in FP64: its own oracle route against the
    # Cholesky reference (CFA eliminates through A, whose conditioning differs from M)
    floors = {a: _rel_err(oracle.fd(model, st.q, st.qdot, st.tau, algo=o, n_threads=8), ref,
                          model.offsets) for a, o in (("abia", "aba"), ("cfa", "cfa"))}
    floors["jsiia"] = floors["abia"]
    floors["cfa_cr"] = floors["cfa_hybrid"] = floors["cfa"]
    for algo, team in (("abia", 1), ("abia", 8), ("abia", 32), ("cfa", 32), ("cfa", 8), ("cfa", 256), ("jsiia", 32),
                       ("jsiia", 128), ("cfa_cr", 1), ("cfa_cr", 32), ("cfa_cr", 256),
                       ("cfa_hybrid", 1), ("cfa_hybrid", 32), ("cfa_hybrid", 256)):
        got, status = _gpu(model, st, algo, "fp64", team)
        assert (status == 0).all(), (algo, team)
        err = _rel_err(got, ref, model.offsets)
        tol = np.maximum(1e-10, 10 * np.maximum(floors[algo], floors["abia"]))
        print(f"n={n} {algo} team {team}: max err {err.max():.2e}, floor {floors[algo].max():.2e}")
        assert (err <= tol).all(), (algo, team, err.max(), tol.min())


def test_uneven_batch_mixed_precision_sampled():
    """2 000 chains, n log-uniform in [6, 512]; FP64 OEE / ABI accumulation with
    FP32 elsewhere; 24 sampled chains against the FP64 oracle."""
    lengths = synth.log_uniform_lengths(2000, 6, 512, seed=0)
    model = synth.random_chains(lengths, seed=1)
    st = synth.random_states(model.n_links_total, seed=2)
    rng = np.random.default_rng(3)
    # 20 random chains and the 4 shortest (the well-conditioned end of the batch)
    sample = np.unique(np.concatenate([rng.choice(model.n_chains, 20, replace=False),
                                       np.argsort(lengths, kind="stable")[:4]]))
    ref = oracle.fd(model, st.q, st.qdot, st.tau, problems=sample)
    off = model.offsets
    idx = np.concatenate([np.arange(off[p], off[p + 1]) for p in sample])
    so = np.concatenate([[0], np.cumsum(lengths[sample])])
    cond = np.array([np.linalg.cond(oracle.mass_matrix(model.chain(p), st.q[off[p]:off[p + 1]]))
                     for p in sample])
    for algo in ("abia", "cfa", "jsiia"):
        got64, status = _gpu(model, st, algo, "fp64", 0)
        assert (status == 0).all() and np.isfinite(got64).all(), algo
        err = _rel_err(got64[idx], ref[idx], so)
        assert np.median(err) < 1e-10, (algo, np.median(err))
        gotm, status = _gpu(model, st, algo, "mixed", 0)
        assert (status == 0).all() and np.isfinite(gotm).all(), algo
        errm = _rel_err(gotm[idx], ref[idx], so)
        # 1e-4 on the well-conditioned chains (cond(M) eps32 <= 1e-4); on all, the
        # forward-error bound of a backward-stable single-precision solve
        good = cond * EPS32 <= 1e-4
        assert good.any()
        assert errm[good].max() < 1e-4, (algo, errm[good].max())
        assert (errm <= np.maximum(1e-4, 4 * cond * EPS32)).all(), (algo, errm.max())


def test_uneven_batch_adjoint_central_differences():
    """Adjoint on an uneven batch (n log-uniform in [6, 512]) on 64 sampled chains:
    (1) against central differences of the FP64 oracle (ABA) with h = 1e-6 along a
    random unit direction per chain; for long chains the rounding of the two
    solves divided by 2h limits that comparison, so its bar is 1e-4;
    (2) against Richardson-extrapolated central differences of the GPU solve at
    h = 1e-4, where rounding is negligible, to 2e-6."""
    import oracle
    from paper_1609_06779_gb300 import fd
    lengths = synth.log_uniform_lengths(400, 6, 512, seed=10)
    model = synth.random_chains(lengths, seed=11)
    st = synth.random_states(model.n_links_total, seed=12)
    cs = fd.ChainSet(model)
    b = fd.Batch(cs)
    rng = np.random.default_rng(13)
    t = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")
    q, qd, tau = t(st.q), t(st.qdot), t(st.tau)
    sample = np.sort(rng.choice(model.n_chains, 64, replace=False))
    mask = np.zeros(model.n_links_total)
    for p in sample:
        mask[model.offsets[p]:model.offsets[p + 1]] = 1.0
    w_np = rng.standard_normal(model.n_links_total) * mask
    w = t(w_np)
    qb, qdb, tb, _ = fd.adjoint(b, q, qd, tau, w, algo="cfa", masses=False)
    base = [st.q, st.qdot, st.tau]
    # each chain's own FP64 solve error against the oracle: numerical derivatives
    # divide it by the step, so it sets the chain's bar (tight when well conditioned)
    qdd = fd.solve(b, q, qd, tau, algo="cfa").cpu().numpy()
    ref = oracle.fd(model, st.q, st.qdot, st.tau, algo="cholesky", problems=sample)
    eps, size = {}, {}
    for p in sample:
        a_, c_ = model.offsets[p], model.offsets[p + 1]
        eps[p] = np.abs(qdd[a_:c_] - ref[a_:c_]).max() / np.abs(ref[a_:c_]).max()
        size[p] = np.abs(w_np[a_:c_] * ref[a_:c_]).sum()   # scale of the terms of <w, qdd>

    def gpu_central(which, d, step):
        args_p = [q, qd, tau]; args_m = [q, qd, tau]
        args_p[which] = args_p[which] + step * d
        args_m[which] = args_m[which] - step * d
        return ((fd.solve(b, *args_p, algo="cfa") - fd.solve(b, *args_m, algo="cfa")) * w
                ).cpu().numpy() / (2 * step)

    worst_oracle = 0.0
    for grad, which in ((qb, 0), (qdb, 1), (tb, 2)):
        d_np = rng.standard_normal(model.n_links_total) * mask
        for p in sample:  # a unit direction per chain
            a_, c_ = model.offsets[p], model.offsets[p + 1]
            d_np[a_:c_] /= np.linalg.norm(d_np[a_:c_])
        d = t(d_np)
        num = (4 * gpu_central(which, d, 5e-5) - gpu_central(which, d, 1e-4)) / 3
        ana = (grad * d).cpu().numpy()
        up = list(base); up[which] = base[which] + 1e-6 * d_np
        dn = list(base); dn[which] = base[which] - 1e-6 * d_np
        orc = (oracle.fd(model, *up, algo="aba", problems=sample)
               - oracle.fd(model, *dn, algo="aba", problems=sample)) / 2e-6
        for p in sample:
            a_, c_ = model.offsets[p], model.offsets[p + 1]
            an = ana[a_:c_].sum()
            n_gpu = num[a_:c_].sum()
            n_orc = w_np[a_:c_] @ orc[a_:c_]
            # rounding of <w, qdd> is about eps * sum|w qdd|; Richardson over h = 1e-4
            # and 5e-5 turns it into at most 3 eps sum|w qdd| / 1e-4
            tol_gpu = 2e-6 * max(abs(n_gpu), 1.0) + 3 * eps[p] * size[p] / 1e-4
            assert abs(an - n_gpu) <= tol_gpu, (which, p, an, n_gpu, tol_gpu)
            rel = abs(an - n_orc) / max(abs(n_orc), 1.0)
            worst_oracle = max(worst_oracle, rel)
            tol_orc = 1e-4 * max(abs(n_orc), 1.0) + 2 * eps[p] * size[p] / 1e-6
            assert abs(an - n_orc) <= tol_orc, (which, p, an, n_orc, tol_orc)
    print(f"adjoint vs oracle central differences (h=1e-6): worst relative {worst_oracle:.2e}")


def test_uneven_batch_mixed_adjoint_central_differences():
    """The mixed-precision adjoint (CFA; FP32 inverse dynamics and reverse sweep,
    FP64 blocks and elimination) on the uneven batch, 64 sampled chains, against
    central differences of the FP64 oracle (ABA, h = 1e-6) along a random unit
    direction per chain. Bar per chain: the single-precision forward-error bound
    max(1e-4, 4 cond(M) eps32) times the size of the gradient (its FP64 adjoint,
    which the FP64 test checks), plus the rounding of the oracle's differences."""
    from paper_1609_06779_gb300 import fd
    lengths = synth.log_uniform_lengths(400, 6, 512, seed=10)
    model = synth.random_chains(lengths, seed=11)
    st = synth.random_states(model.n_links_total, seed=12)
    cs = fd.ChainSet(model)
    b = fd.Batch(cs)
    rng = np.random.default_rng(13)
    sample = np.sort(rng.choice(model.n_chains, 64, replace=False))
    mask = np.zeros(model.n_links_total)
    for p in sample:
        mask[model.offsets[p]:model.offsets[p + 1]] = 1.0
    w_np = rng.standard_normal(model.n_links_total) * mask
    t64 = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")
    t32 = lambda a: torch.tensor(a, dtype=torch.float32, device="cuda")
    g32 = fd.adjoint(b, t32(st.q), t32(st.qdot), t32(st.tau), t32(w_np), algo="cfa",
                     prec="mixed", masses=False)
    g64 = fd.adjoint(b, t64(st.q), t64(st.qdot), t64(st.tau), t64(w_np), algo="cfa",
                     masses=False)
    ref = oracle.fd(model, st.q, st.qdot, st.tau, algo="cholesky", problems=sample)
    aba = oracle.fd(model, st.q, st.qdot, st.tau, algo="aba", problems=sample)
    cond, eps64, size = {}, {}, {}
    for p in sample:
        a_, c_ = model.offsets[p], model.offsets[p + 1]
        cond[p] = np.linalg.cond(oracle.mass_matrix(model.chain(p), st.q[a_:c_]))
        eps64[p] = max(np.abs(aba[a_:c_] - ref[a_:c_]).max() / np.abs(ref[a_:c_]).max(), 1e-16)
        size[p] = np.abs(w_np[a_:c_] * ref[a_:c_]).sum()
    base = [st.q, st.qdot, st.tau]
    n_good = 0
    for which in range(3):
        d_np = rng.standard_normal(model.n_links_total) * mask
        for p in sample:
            a_, c_ = model.offsets[p], model.offsets[p + 1]
            d_np[a_:c_] /= np.linalg.norm(d_np[a_:c_])
        up = list(base); up[which] = base[which] + 1e-6 * d_np
        dn = list(base); dn[which] = base[which] - 1e-6 * d_np
        orc = (oracle.fd(model, *up, algo="aba", problems=sample)
               - oracle.fd(model, *dn, algo="aba", problems=sample)) / 2e-6
        ana = (g32[which].double() * t64(d_np)).cpu().numpy()
        gn = g64[which].cpu().numpy()
        for p in sample:
            a_, c_ = model.offsets[p], model.offsets[p + 1]
            n_orc = w_np[a_:c_] @ orc[a_:c_]
            an = ana[a_:c_].sum()
            rel = max(1e-4, 4 * cond[p] * EPS32)
            tol = rel * np.linalg.norm(gn[a_:c_]) + 1e-4 * max(abs(n_orc), 1.0) \
                + 2 * eps64[p] * size[p] / 1e-6
            assert abs(an - n_orc) <= tol, (which, p, lengths[p], an, n_orc, tol)
            n_good += cond[p] * EPS32 <= 1e-4
    assert n_good > 0
