"""fd_solve_cfa_static: CFA with the library's static scratch instead of a
caller workspace, for callers that must not allocate device memory when they
solve (a control loop with a hard deadline, a host callback, a framework that
owns all device memory). Called through the C ABI.

Both entry points run the same kernel with the same team on the same inputs, so
their results must be equal bit for bit; two calls in a row check that the
second call does not depend on what the first left in the shared scratch. The
FP64 result is also checked against the oracle. Kept in its own file, collected
last."""
import ctypes

import numpy as np
import pytest

from paper_1609_06779_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

LENGTHS = [32] * 300 + [7, 1, 13, 0, 64]


def _setup(prec):
    from paper_1609_06779_gb300 import fd
    model = synth.random_chains(LENGTHS, seed=31)
    st = synth.random_states(model.n_links_total, seed=32)
    cs = fd.ChainSet(model)
    dt = torch.float64 if prec == "fp64" else torch.float32
    q, qd, tau = (torch.tensor(x, dtype=dt, device="cuda") for x in (st.q, st.qdot, st.tau))
    return fd, model, st, cs, q, qd, tau


def _static(lib, fd, cs, q, qd, tau, prec, team, stream):
    out = torch.full_like(q, float("nan"))
    status = torch.full((cs.info()[0],), -1, dtype=torch.int32, device="cuda")
    rc = lib.fd_solve_cfa_static(cs.handle, q.data_ptr(), qd.data_ptr(), tau.data_ptr(),
                                 out.data_ptr(), fd.PRECS[prec], team, status.data_ptr(),
                                 ctypes.c_void_p(stream.cuda_stream))
    assert rc == 0, lib.fd_last_error()
    stream.synchronize()
    return out, status


@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp32"])
@pytest.mark.parametrize("team", [32, 0])
def test_static_scratch_cfa_equals_workspace_cfa(prec, team):
    fd, model, st, cs, q, qd, tau = _setup(prec)
    lib = fd.load()
    b = fd.Batch(cs)  # problem p = chain p, untuned
    # team 0: the documented default, the largest power of two not above
    # 152 x 2048 / n_chains, capped at the longest chain rounded up to a power of two
    expect = team
    if team == 0:
        expect = 1
        while 2 * expect <= 152 * 2048 // len(LENGTHS) and expect < 256:
            expect *= 2
        cap = 1
        while cap < max(LENGTHS) and cap < 256:
            cap *= 2
        expect = min(expect, cap)
    ref = fd.solve(b, q, qd, tau, algo="cfa", prec=prec, team=expect)
    torch.cuda.synchronize()
    # a non-blocking side stream: nothing orders the solve after work on the legacy stream
    stream = torch.cuda.Stream(priority=0)
    for call in range(2):
        out, status = _static(lib, fd, cs, q, qd, tau, prec, team, stream)
        assert (status.cpu().numpy() == 0).all(), call
        assert torch.equal(out, ref), (call, (out - ref).abs().max().item())


def test_static_scratch_cfa_matches_oracle():
    import oracle
    fd, model, st, cs, q, qd, tau = _setup("fp64")
    lib = fd.load()
    out, status = _static(lib, fd, cs, q, qd, tau, "fp64", 0, torch.cuda.current_stream())
    assert (status.cpu().numpy() == 0).all()
    got = out.cpu().numpy()
    ref = oracle.fd(model, st.q, st.qdot, st.tau, algo="cholesky")
    aba = oracle.fd(model, st.q, st.qdot, st.tau, algo="aba")
    for p in range(len(LENGTHS)):
        a, z = model.offsets[p], model.offsets[p + 1]
        if z == a:
            continue
        scale = max(np.abs(ref[a:z]).max(), 1e-300)
        floor = np.abs(aba[a:z] - ref[a:z]).max() / scale  # the oracle's own FP64 floor
        err = np.abs(got[a:z] - ref[a:z]).max() / scale
        assert err <= max(1e-10, 10 * floor), (p, err, floor)


def test_static_scratch_wrapper_and_limits():
    from paper_1609_06779_gb300 import fd
    lib = fd.load()
    model = synth.random_chains([32] * 1000, seed=1)    # 32 000 links: above the limit
    cs = fd.ChainSet(model)
    x = torch.zeros(model.n_links_total, dtype=torch.float64, device="cuda")
    rc = lib.fd_solve_cfa_static(cs.handle, x.data_ptr(), x.data_ptr(), x.data_ptr(),
                                 x.data_ptr(), 0, 0, None, None)
    assert rc == 1
    assert b"static scratch" in lib.fd_last_error()
    # a team the kernels are not built for
    small = fd.ChainSet(synth.random_chains([5, 6], seed=2))
    y = torch.zeros(11, dtype=torch.float64, device="cuda")
    assert lib.fd_solve_cfa_static(small.handle, y.data_ptr(), y.data_ptr(), y.data_ptr(),
                                   y.data_ptr(), 0, 3, None, None) == 1
    # the binding checks the output and status arrays before the call
    with pytest.raises(fd.FDError):
        fd.solve_cfa_static(small, y, y, y, out=torch.zeros(10, dtype=torch.float64,
                                                              device="cuda"))
    with pytest.raises(fd.FDError):
        fd.solve_cfa_static(small, y, y, y,
                            status=torch.zeros(1, dtype=torch.int32, device="cuda"))
    out = fd.solve_cfa_static(small, y, y, y)
    torch.cuda.synchronize()
    assert torch.isfinite(out).all()
