"""fd_solve_cfa_static: CFA with the library's static scratch instead of a
caller workspace, for callers that must not allocate device memory when they
solve. Called through the C ABI; compared with fd_solve_batch (CFA), two calls
in a row (the second reuses the scratch the first left behind). Kept in its own
file, collected last."""
import ctypes

import numpy as np
import pytest

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


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 1e-4)])
def test_static_scratch_cfa_matches_workspace_cfa(prec, tol):
    from paper_1609_06779_gb300 import fd
    lib = fd.load()
    model = synth.random_chains([32] * 300 + [7, 1, 13, 0, 64], seed=31)
    st = synth.random_states(model.n_links_total, seed=32)
    cs = fd.ChainSet(model)
    b = fd.Batch(cs)
    dt = torch.float64 if prec == "fp64" else torch.float32
    q, qd, tau = (torch.tensor(x, dtype=dt, device="cuda") for x in (st.q, st.qdot, st.tau))
    # the same team on both sides, so the two entry points run the same arithmetic
    team = 32
    ref = fd.solve(b, q, qd, tau, algo="cfa", prec=prec, team=team).double().cpu().numpy()
    stream = torch.cuda.current_stream()
    for call in range(2):
        out = torch.full_like(q, float("nan"))
        status = torch.full((cs.info()[0],), -1, dtype=torch.int32, device="cuda")
        rc = lib.fd_solve_cfa_static(cs.handle, q.data_ptr(), qd.data_ptr(), tau.data_ptr(),
                                     out.data_ptr(), fd.PRECS[prec], team, status.data_ptr(),
                                     ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0, lib.fd_last_error()
        torch.cuda.synchronize()
        got = out.double().cpu().numpy()
        assert np.isfinite(got).all(), call
        assert (status.cpu().numpy() == 0).all(), call
        assert _rel_err(got, ref, model.offsets).max() <= tol, call


def test_static_scratch_rejects_oversize_sets():
    from paper_1609_06779_gb300 import fd
    lib = fd.load()
    model = synth.random_chains([32] * 1000, seed=1)    # 32 000 links: above the limit
    cs = fd.ChainSet(model)
    x = torch.zeros(model.n_links_total, dtype=torch.float64, device="cuda")
    rc = lib.fd_solve_cfa_static(cs.handle, x.data_ptr(), x.data_ptr(), x.data_ptr(),
                                 x.data_ptr(), 0, 0, None, None)
    assert rc == 1
    assert b"static scratch" in lib.fd_last_error()
