"""Batch partitioning across ranks, on CPU with the gloo backend (world size 2):
the shards cover the batch exactly once, the timing reductions and the gather
of per-rank results (the oracle's qdd of each rank's chains) behave as the
benchmark's multi-GPU path expects."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1609_06779_gb300 import dist as fdist  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_1609_06779_gb300 import synth
        r, w, _ = fdist.env()
        n_chains = 9
        a, b = fdist.shard(n_chains, r, w)
        model = synth.random_chains([3, 4, 5, 6, 3, 4, 5, 6, 7], seed=0)
        sub = synth.ChainModel(model.axes[model.offsets[a]:model.offsets[b]],
                               model.frames[model.offsets[a]:model.offsets[b]],
                               model.inertias[model.offsets[a]:model.offsets[b]],
                               model.offsets[a:b + 1] - model.offsets[a], model.gravity)
        st = synth.random_states(model.n_links_total, seed=1)
        sl = slice(model.offsets[a], model.offsets[b])
        qdd = oracle.fd(sub, st.q[sl], st.qdot[sl], st.tau[sl])
        t_max = fdist.max_over_ranks(10.0 + r)
        total = fdist.sum_over_ranks(b - a)
        got = fdist.gather_to_rank0(torch.tensor(qdd))
        if r == 0:
            full = oracle.fd(model, st.q, st.qdot, st.tau)
            q.put(("ok", t_max, total, float(np.abs(got.numpy() - full).max())))
    except Exception as e:  # pragma: no cover
        q.put(("err", repr(e)))
        raise
    finally:
        dist.destroy_process_group()


def test_shards_cover_batch():
    for n in (0, 1, 7, 65536):
        for w in (1, 2, 3, 8):
            spans = [fdist.shard(n, r, w) for r in range(w)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(spans[i][1] == spans[i + 1][0] for i in range(w - 1))
            sizes = [b - a for a, b in spans]
            assert max(sizes) - min(sizes) <= 1


def test_two_rank_gloo_partition_and_gather():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
    assert res[0] == "ok", res
    _, t_max, total, err = res
    assert t_max == 11.0 and total == 9.0
    assert err == 0.0
