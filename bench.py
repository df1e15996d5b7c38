"""Benchmark: batched forward dynamics of 65 536 independent 32-link chains.

One step = ABIA, JSIIA and CFA each solving the whole batch in FP64 (3 x 65 536
FD solves) through the C ABI, inputs resident on the device. Prints one JSON
line (rank 0). ``--impl reference`` times the FP64 CPU oracle instead.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1609_06779_gb300 import dist as fdist  # noqa: E402
from paper_1609_06779_gb300 import roofline, synth  # noqa: E402

N_CHAINS = 65536
N_LINKS = 32
ALGOS = ("abia", "jsiia", "cfa")
METRIC = "FD solves/s (32-link, batch 64K) ABIA/JSIIA/CFA"
WORKLOAD = "65536 independent 32-link revolute chains (random models, seed 0), FP64"
# GB300 FP64 (152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz): replaced at run time by
# the rate measured on this GPU (fd_measure_fp64_peak), see measure_peak()
FP64_PEAK_TFLOPS = 1.25
PEAK_INFO = {"source": "nominal (not measured)"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--chains", type=int, default=N_CHAINS)
    ap.add_argument("--links", type=int, default=N_LINKS)
    ap.add_argument("--teams", default="",
                    help="fixed teams, e.g. abia=1,jsiia=8,cfa=16,cfa_cr=4 (others autotuned)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-extra", action="store_true")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the context variants (CR, hybrid, ID, adjoint, FP32, mixed)")
    ap.add_argument("--no-peak", action="store_true",
                    help="do not measure the FP64 peak (report against the nominal 1.25 TFLOP/s)")
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--serve-rate", type=float, default=20000.0)
    return ap.parse_args()


def fixed_teams(spec: str) -> dict:
    out = {}
    for item in filter(None, spec.split(",")):
        k, v = item.split("=")
        out[k.strip()] = int(v)
    return out


def dist_env():
    return fdist.env()


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, path, index):
        self.path, self.proc = path, None
        self.index = index

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        except Exception:
            rows = []
        rows = [[c.strip() for c in r] for r in rows if len(r) >= 9]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def traffic_record(kernel: str, team: int):
    """DRAM bytes per link of `kernel` at `team` from the committed ncu summary,
    if the kernel sources are unchanged since the capture."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        rec = json.load(open(path))
        ent = rec[kernel][str(team)]
    except Exception:
        return None
    if rec.get("csrc_sha") != csrc_sha():
        return None
    return ent


def measure_peak(fd, device):
    """The FP64 roofline denominator, measured on this GPU: independent DFMA
    chains (fd_measure_fp64_peak), best of three runs of a few hundred
    milliseconds, with the SM clock sampled meanwhile."""
    global FP64_PEAK_TFLOPS, PEAK_INFO
    clk = Clocks(os.path.join(tempfile.gettempdir(), f"fd_peak_clocks_{os.getpid()}.csv"), device)
    runs = []
    with clk:
        time.sleep(0.3)
        for _ in range(3):
            runs.append(fd.measure_fp64_peak(device, 200000))
    best = max(r[0] for r in runs)
    cs = clk.summary()
    FP64_PEAK_TFLOPS = best
    PEAK_INFO = {"source": "measured: fd_measure_fp64_peak (independent DFMA chains, 4 blocks x "
                           "128 threads per SM), best of 3",
                 "tflops_runs": [r[0] for r in runs], "ms_runs": [r[1] for r in runs],
                 "clocks": cs,
                 "tflops_at_max_clock": (best * cs["sm_max_mhz"] / cs["sm_mhz"]
                                         if cs.get("sm_mhz") and cs.get("sm_max_mhz") else None)}
    return best


def measured_hbm_gbs():
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except Exception:
        return None


def csrc_sha() -> str:
    """Hash of the sources the forward-dynamics kernels are compiled from (their
    headers and launch units), so a traffic record stays valid only for them."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1609_06779_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        if f in ("fd_layout.h", "fd_device.cuh", "fd_kernels.cuh", "fd_launch.h") or (
                f.startswith(("k_abia", "k_jsiia", "k_cfa")) and f.endswith(".cu")):
            h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def cpu_oracle(model, st, n_problems, budget_s=10.0, threads=None):
    """Time the FP64 CPU oracle (the three algorithms) on a bounded sample."""
    import oracle
    threads = threads or os.cpu_count() or 1
    n = int(model.offsets[1] - model.offsets[0])
    sample = min(n_problems, 4096)
    # the first `sample` chains as their own model
    L = sample * n
    sub = synth.ChainModel(model.axes[:L], model.frames[:L], model.inertias[:L],
                           model.offsets[:sample + 1].copy(), model.gravity)
    q, qd, tau = st.q[:L], st.qdot[:L], st.tau[:L]
    algos = {"abia": "aba", "jsiia": "cholesky", "cfa": "cfa"}
    t0 = time.perf_counter()
    solved = 0
    while True:
        for a in ALGOS:
            oracle.fd(sub, q, qd, tau, algo=algos[a], n_threads=threads)
            solved += sample
        el = time.perf_counter() - t0
        if el > budget_s:
            break
    # the same sample on one core, for a shorter budget
    t1 = time.perf_counter()
    one = 0
    while True:
        for a in ALGOS:
            oracle.fd(sub, q, qd, tau, algo=algos[a], n_threads=1)
            one += sample
        el1 = time.perf_counter() - t1
        if el1 > budget_s / 3:
            break
    return {"value": solved / el, "unit": "FD solves/s", "cores": threads, "kind": "oracle",
            "value_1core": one / el1,
            "sample": f"first {sample} of {n_problems} chains x {{ABA, Cholesky (JSIIA), CFA+OEE}},"
                      f" {solved} solves in {el:.1f} s on {threads} cores (OpenMP across chains),"
                      f" {one} in {el1:.1f} s on one core, FP64"}


def accuracy(model, st, outs, sample32=4096):
    """Largest error per chain, max |qdd - ref| / max(max |ref|, 1), of each output
    against the FP64 oracle (dense Cholesky): every chain for the FP64 paths, the
    first `sample32` chains for the FP32 and mixed paths (also against the oracle
    fed the same states rounded to FP32)."""
    import oracle
    n = int(model.offsets[1] - model.offsets[0])
    threads = os.cpu_count() or 1
    f32 = lambda a: a.astype(np.float32).astype(np.float64)
    K = model.n_chains
    ref = oracle.fd(model, st.q, st.qdot, st.tau, algo="cholesky",
                    n_threads=threads).reshape(K, n)
    k32 = min(sample32, K)
    L32 = k32 * n
    sub = synth.ChainModel(model.axes[:L32], model.frames[:L32], model.inertias[:L32],
                           model.offsets[:k32 + 1].copy(), model.gravity)
    ref32 = oracle.fd(sub, f32(st.q[:L32]), f32(st.qdot[:L32]), f32(st.tau[:L32]),
                      algo="cholesky", n_threads=threads).reshape(k32, n)
    # cond(M) of the sampled chains: a backward-stable single-precision solve
    # loses about cond(M) eps32; "well conditioned" means cond(M) eps32 <= 1e-4
    eps32 = float(np.finfo(np.float32).eps)
    cond = np.array([np.linalg.cond(oracle.mass_matrix(model.chain(k),
                                                       st.q[model.offsets[k]:model.offsets[k + 1]]))
                     for k in range(k32)])
    res = {"reference": "FP64 CPU oracle, dense Cholesky", "chains_fp64": K,
           "chains_float": k32, "float_paths_also_vs_states_rounded_to_fp32": {},
           "cond_M_float_sample": {"min": float(cond.min()), "median": float(np.median(cond)),
                                   "max": float(cond.max()),
                                   "well_conditioned_chains": int((cond * eps32 <= 1e-4).sum())},
           "float_err_over_cond_eps32_max": {}}

    def errs(got, r):
        scale = np.maximum(np.abs(r).max(axis=1), 1.0)
        return np.abs(got - r).max(axis=1) / scale
    for k, v in outs.items():
        got = v.double().numpy()
        rows = got.size // n
        got = got.reshape(rows, n)
        res[k] = float(errs(got, ref[:rows]).max())
        if not k.endswith("fp64"):
            e32 = errs(got[:k32], ref[:k32])
            res["float_paths_also_vs_states_rounded_to_fp32"][k] = float(errs(got[:k32], ref32).max())
            res["float_err_over_cond_eps32_max"][k] = float((e32 / (cond * eps32)).max())
    return res


def serve_bench(seconds=10.0, rate=20000.0, per_size=False, budget=40 << 30, seed=0,
                device=0):
    """Open-loop Poisson stream of FD+gradient queries and 50-step rollouts
    (dt = 1e-3) on chains of 6..256 links (log-uniform), 50/50; latency =
    completion - scheduled arrival."""
    from paper_1609_06779_gb300 import fd
    rng = np.random.default_rng(seed)
    n_models, n_templates, steps = 1024, 2048, 50
    lengths = synth.log_uniform_lengths(n_models, 6, 256, seed=seed)
    models = synth.random_chains(lengths, seed=seed + 1)
    srv = fd.Server(device=device, budget_bytes=budget, per_size=per_size)
    ids = [srv.add_model(models.chain(k)) for k in range(n_models)]
    temps = []
    for j in range(n_templates):
        k = int(rng.integers(n_models))
        n = int(lengths[k])
        q = rng.uniform(-np.pi, np.pi, n)
        qd = rng.standard_normal(n)
        if j % 2 == 0:
            temps.append((0, ids[k], n, q, qd, rng.standard_normal(n) * 10, rng.standard_normal(n)))
        else:
            temps.append((1, ids[k], n, q, qd, rng.standard_normal((steps, n)) * 10, None))
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=int(rate * seconds * 1.2) + 16))
    arrivals = arrivals[arrivals < seconds]
    sched, kinds, links = {}, {}, {}
    lat = {0: [], 1: []}
    t0 = fd.serve_clock() + 0.05
    k = 0
    n_total = len(arrivals)
    busy_refused = 0

    def collect():
        tk, _, done, st = srv.drain()
        for t, d in zip(tk.tolist(), done.tolist()):
            lat[kinds.pop(t)].append(d - sched.pop(t))

    while k < n_total:
        now = fd.serve_clock() - t0
        while k < n_total and arrivals[k] <= now:
            kind, mid, n, q, qd, tau, w = temps[k % n_templates]
            try:
                if kind == 0:
                    t = srv.submit_grad(mid, q, qd, tau, w, algo="cfa")
                else:
                    t = srv.submit_rollout(mid, q, qd, tau, 1e-3, algo="abia")
            except fd.FDError:
                busy_refused += 1
                k += 1
                continue
            sched[t] = t0 + arrivals[k]
            kinds[t] = kind
            k += 1
        collect()
        if k < n_total:
            time.sleep(max(0.0, min(0.0005, arrivals[k] - (fd.serve_clock() - t0))))
    t_end_arrivals = fd.serve_clock()
    while sched and fd.serve_clock() - t_end_arrivals < 120:
        collect()
        time.sleep(0.001)
    st = srv.stats()
    srv.close()
    span = max(fd.serve_clock() - t0, 1e-9)
    out = {"rate_offered": rate, "seconds": seconds, "requests": n_total,
           "refused": busy_refused, "unfinished": len(sched),
           "per_size_launches": per_size, "ticks": st["ticks"], "launches": st["launches"],
           "fd_solves_per_s": (len(lat[0]) + steps * len(lat[1])) / span,
           "link_solves_per_s": st["link_solves"] / span,
           "gpu_busy_frac": st["busy_seconds"] / span}
    for kind, name in ((0, "fd_grad"), (1, "rollout50")):
        v = np.array(lat[kind]) * 1e3
        if len(v):
            out[name] = {"n": int(len(v)), "p50_ms": float(np.percentile(v, 50)),
                         "p99_ms": float(np.percentile(v, 99)), "max_ms": float(v.max())}
    return out


def occupancy(n_problems: int, team: int) -> dict:
    """Warps a launch runs and how many fall on each of the 608 SM sub-partitions
    (152 SMs x 4): below one, the batch is latency-bound, not throughput-bound."""
    warps = -(-n_problems * team // 32)
    return {"warps": warps, "warps_per_subpartition": warps / 608.0}


def _time_ms(fn, reps=3, warm=1):
    import torch
    for _ in range(warm):
        fn()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def extra_configs(dev, keep=None):
    """The paper-shaped workloads besides the headline batch: one 7-link chain
    with 1024 states (launch-bound; CUDA-graph replay), long chains (256 x 256,
    64 x 1024) and an uneven batch of 100 000 chains (6..512 links, mixed
    precision) as one launch against one launch per distinct length. Appends to
    `keep` a sample of each configuration's results for the accuracy check of
    the CPU leg."""
    keep = [] if keep is None else keep
    import torch
    from paper_1609_06779_gb300 import fd
    t64 = lambda a: torch.tensor(a, dtype=torch.float64, device=dev)
    res = {}

    # 1 chain x 7 links, 1024 states (shared model), FP64
    m = synth.random_chains([7], seed=0)
    ci, so1 = synth.replicate_model(m, 1024)
    st = synth.random_states(7 * 1024, seed=1)
    cs = fd.ChainSet(m, device=dev.index or 0)
    b = fd.Batch(cs, ci)
    q, qd, tau = t64(st.q), t64(st.qdot), t64(st.tau)
    r1 = {}
    k1 = {"config": "1x7_links_1024_states_fp64", "model": m, "chain_index": ci,
          "state_offsets": so1, "st": st, "problems": None, "outs": {}}
    for a in ALGOS + ("cfa_cr", "cfa_hybrid", "abia_scan"):
        team = fd.autotune(b, q, qd, tau, algo=a)
        ws = fd.workspace(b, a, "fp64", 0, dev)
        out = torch.empty_like(q)
        launch_us = 1e3 * _time_ms(lambda: fd.solve(b, q, qd, tau, algo=a, out=out, ws=ws), 50, 5)
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream(device=dev)
        s.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(s):
            fd.solve(b, q, qd, tau, algo=a, out=out, ws=ws)
        torch.cuda.current_stream(dev).wait_stream(s)
        with torch.cuda.graph(g):
            fd.solve(b, q, qd, tau, algo=a, out=out, ws=ws)
        graph_us = 1e3 * _time_ms(g.replay, 50, 5)
        k1["outs"][a] = out.cpu().numpy()
        r1[a] = {"team": team, "launch_us": launch_us, "graph_replay_us": graph_us,
                 "solves_per_s": 1024 / (graph_us * 1e-6), "occupancy": occupancy(1024, team)}
    res["1x7_links_1024_states_fp64"] = r1
    keep.append(k1)
    del cs, b

    # long chains, FP64
    for n, count in ((256, 256), (1024, 64)):
        m = synth.random_chains([n] * count, seed=n)
        st = synth.random_states(m.n_links_total, seed=n + 1)
        cs = fd.ChainSet(m, device=dev.index or 0)
        b = fd.Batch(cs)
        q, qd, tau = t64(st.q), t64(st.qdot), t64(st.tau)
        rl = {}
        kl = {"config": f"{count}x{n}_links_fp64", "model": m, "chain_index": None, "st": st,
              "problems": [0, 1] if n <= 256 else [0], "outs": {}}
        for a in ALGOS + ("cfa_cr", "cfa_hybrid", "abia_scan"):
            # JSIIA is cubic in n: at 1 024 links one timed solve, no autotuning
            team = 128 if a == "jsiia" else fd.autotune(b, q, qd, tau, algo=a)
            ws = fd.workspace(b, a, "fp64", team, dev)
            out = torch.empty_like(q)
            reps = (1, 1) if (a == "jsiia" and n > 256) else (3, 1)
            ms = _time_ms(lambda: fd.solve(b, q, qd, tau, algo=a, team=team, out=out, ws=ws),
                          *reps)
            kl["outs"][a] = out.cpu().numpy()
            fl = roofline.flops(a, [n] * count)
            rl[a] = {"team": team, "ms": ms, "solves_per_s": count / (ms * 1e-3),
                     "occupancy": occupancy(count, team),
                     "tflops": fl / (ms * 1e-3) / 1e12,
                     "frac_fp64_peak": fl / (ms * 1e-3) / 1e12 / FP64_PEAK_TFLOPS}
        res[f"{count}x{n}_links_fp64"] = rl
        keep.append(kl)
        del cs, b, q, qd, tau
        torch.cuda.empty_cache()

    # uneven batch: 100 000 chains, n log-uniform in [6, 512], mixed precision:
    # one launch split by length class (a team per class, autotuned per class),
    # timed eagerly and as a CUDA-graph replay, against the best single team for
    # the whole batch and against one launch per distinct length
    lengths = synth.log_uniform_lengths(100000, 6, 512, seed=0)
    m = synth.random_chains(lengths, seed=1)
    st = synth.random_states(m.n_links_total, seed=2)
    cs = fd.ChainSet(m, device=dev.index or 0)
    b = fd.Batch(cs)
    t32 = lambda a: torch.tensor(a, dtype=torch.float32, device=dev)
    q, qd, tau = t32(st.q), t32(st.qdot), t32(st.tau)
    ru = {"chains": 100000, "links": int(m.n_links_total), "prec": "mixed"}
    ku = {"config": "100000_uneven_6_512_mixed", "model": m, "chain_index": None, "st": st,
          "problems": np.random.default_rng(5).choice(100000, 64, replace=False).tolist(),
          "outs": {}}
    for a in ("abia", "cfa", "cfa_cr", "cfa_hybrid"):
        fd.autotune(b, q, qd, tau, algo=a, prec="mixed")   # per length class
        classes = fd.batch_classes(b, a, "mixed")
        ws = fd.workspace(b, a, "mixed", 0, dev)
        out = torch.empty_like(q)
        one_ms = _time_ms(lambda: fd.solve(b, q, qd, tau, algo=a, prec="mixed", out=out, ws=ws))
        s_cap = torch.cuda.Stream(device=dev)
        s_cap.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(s_cap):
            fd.solve(b, q, qd, tau, algo=a, prec="mixed", out=out, ws=ws)
        torch.cuda.current_stream(dev).wait_stream(s_cap)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            fd.solve(b, q, qd, tau, algo=a, prec="mixed", out=out, ws=ws)
        graph_ms = _time_ms(g.replay)
        torch.cuda.synchronize()
        ku["outs"][a + "_mixed"] = out.double().cpu().numpy()
        del g
        # one team for every chain (the schedule without length classes)
        single = {}
        for tm in ((1, 8, 32) if a == "abia" else (4, 8, 16, 32)):
            single[tm] = _time_ms(lambda: fd.solve(b, q, qd, tau, algo=a, prec="mixed", team=tm,
                                                   out=out, ws=ws))
        best_t = min(single, key=single.get)
        del ws
        # one launch per distinct chain length (static batching per size)
        groups = []
        off = m.offsets
        for ln in np.unique(lengths):
            idx = np.nonzero(lengths == ln)[0].astype(np.int32)
            links = np.concatenate([np.arange(off[i], off[i + 1]) for i in idx])
            li = torch.tensor(links, device=dev)
            bb = fd.Batch(cs, idx)
            groups.append((bb, q[li].contiguous(), qd[li].contiguous(), tau[li].contiguous(),
                           torch.empty(len(links), dtype=torch.float32, device=dev),
                           fd.workspace(bb, a, "mixed", 0, dev)))

        def per_size():
            for bb, gq, gqd, gtau, go, gw in groups:
                fd.solve(bb, gq, gqd, gtau, algo=a, prec="mixed", out=go, ws=gw)

        ps_ms = _time_ms(per_size)
        ru[a] = {"classes": [{"links": f"{c['min_len']}-{c['max_len']}", "chains": c["count"],
                              "team": c["team"]} for c in classes],
                 "one_launch_ms": one_ms, "graph_replay_ms": graph_ms,
                 "single_team_ms": {str(k): v for k, v in single.items()},
                 "best_single_team": best_t,
                 "per_size_launches_ms": ps_ms, "per_size_launches": len(groups),
                 "solves_per_s_graph": 100000 / (graph_ms * 1e-3),
                 "solves_per_s_one_launch": 100000 / (one_ms * 1e-3),
                 "solves_per_s_best_single_team": 100000 / (single[best_t] * 1e-3),
                 "solves_per_s_per_size": 100000 / (ps_ms * 1e-3),
                 "gflop": roofline.flops(a, lengths) / 1e9,
                 "tflops_graph": roofline.flops(a, lengths) / (graph_ms * 1e-3) / 1e12}
        del groups
        torch.cuda.empty_cache()
    w = torch.randn(m.n_links_total, dtype=torch.float32, device=dev)
    fd.autotune(b, q, qd, tau, algo="cfa", prec="mixed")
    adj_ms = _time_ms(lambda: fd.adjoint(b, q, qd, tau, w, algo="cfa", prec="mixed",
                                         masses=False))
    ru["adjoint_cfa_ms"] = adj_ms
    ru["adjoint_solves_per_s"] = 100000 / (adj_ms * 1e-3)
    res["100000_uneven_6_512_mixed"] = ru
    keep.append(ku)
    del cs, b, q, qd, tau, w
    torch.cuda.empty_cache()

    # kinematic trees (fd_create_tree; branched robots, beyond the paper's serial
    # chains): 65 536 random trees of 32 links, ABIA and JSIIA over the parent
    # array, one thread per tree, FP64; the first 256 trees against the oracle
    m = synth.random_trees([32] * 65536, seed=0)
    st = synth.random_states(m.n_links_total, seed=1000)
    cs = fd.ChainSet(m, device=dev.index or 0)
    b = fd.Batch(cs)
    q, qd, tau = t64(st.q), t64(st.qdot), t64(st.tau)
    local = np.concatenate([np.arange(32) - 1] * 65536)
    rt = {"trees": 65536, "links": 32,
          "branching_links": int((m.parents != local).sum()),
          "links_on_the_base": int((m.parents < 0).sum())}
    kt = {"config": "65536_trees_32_links_fp64", "model": m, "st": st, "tree": True,
          "chain_index": None, "problems": list(range(256)), "outs": {}}
    for a in ("abia", "jsiia"):
        ws = fd.workspace(b, a, "fp64", 1, dev)
        out = torch.empty_like(q)
        ms = _time_ms(lambda: fd.solve(b, q, qd, tau, algo=a, out=out, ws=ws), 5, 2)
        kt["outs"][a] = out[:256 * 32].cpu().numpy()
        rt[a] = {"team": 1, "ms": ms, "solves_per_s": 65536 / (ms * 1e-3)}
        del ws, out
    res["65536_trees_32_links_fp64"] = rt
    keep.append(kt)
    del cs, b, q, qd, tau
    torch.cuda.empty_cache()

    # the same trees closed by one revolute loop joint each (fd_tree_add_loops):
    # JSIIA with the constrained solve, FP64; the first 64 against the oracle's
    # dense KKT solve
    loops = synth.random_loops(m, per_tree=1, seed=1)
    cs = fd.ChainSet(m, device=dev.index or 0)
    cs.add_loops(loops)
    b = fd.Batch(cs)
    q, qd, tau = t64(st.q), t64(st.qdot), t64(st.tau)
    ws = fd.workspace(b, "jsiia", "fp64", 1, dev)
    out = torch.empty_like(q)
    ms = _time_ms(lambda: fd.solve(b, q, qd, tau, algo="jsiia", out=out, ws=ws), 5, 2)
    res["65536_looped_trees_32_links_fp64"] = {
        "trees": 65536, "links": 32, "loops_per_tree": 1, "algo": "jsiia", "team": 1, "ms": ms,
        "solves_per_s": 65536 / (ms * 1e-3)}
    keep.append({"config": "65536_looped_trees_32_links_fp64", "model": m, "st": st,
                 "tree": True, "loops": loops, "chain_index": None, "problems": list(range(64)),
                 "outs": {"jsiia": out[:64 * 32].cpu().numpy()}})
    del cs, b, q, qd, tau, ws, out
    return res


def config_accuracy(keep):
    """Per configuration and path: the largest error per problem,
    max |qdd - ref| / max(max |ref|, 1), on the sampled problems against the FP64
    oracle's dense Cholesky, beside the oracle's own ABA on the same problems (the
    FP64 floor those chains allow)."""
    import oracle
    out = {}
    for k in keep:
        m, st = k["model"], k["st"]
        if k.get("tree"):
            # kinematic trees: the oracle's dense definitions over the parent
            # array (one route, one core) on the first sampled trees
            probs = k["problems"]
            z = int(m.offsets[len(probs)])
            sub = synth.ChainModel(m.axes[:z], m.frames[:z], m.inertias[:z],
                                   m.offsets[:len(probs) + 1].copy(), m.gravity, m.parents[:z])
            t0 = time.perf_counter()
            if k.get("loops") is not None:
                lp = k["loops"]
                sel = np.asarray(lp["tree"]) < len(probs)
                ref = oracle.fd_looped(sub, st.q[:z], st.qdot[:z], st.tau[:z],
                                       {kk: np.asarray(v)[sel] for kk, v in lp.items()})
            else:
                ref = oracle.fd_tree(sub, st.q[:z], st.qdot[:z], st.tau[:z])
            t1 = time.perf_counter()
            r = {"sampled_problems": len(probs),
                 "cpu_oracle": {"kind": "oracle (dense definitions over the parent array)",
                                "cores": 1, "problems": len(probs),
                                "dense_solves_per_s": len(probs) / max(t1 - t0, 1e-9),
                                "sample": f"the first {len(probs)} of {m.n_chains} trees, FP64"}}
            for name, x in k["outs"].items():
                e = 0.0
                for p in range(len(probs)):
                    a, b = int(m.offsets[p]), int(m.offsets[p + 1])
                    e = max(e, float(np.abs(x[a:b] - ref[a:b]).max()
                                     / max(np.abs(ref[a:b]).max(), 1.0)))
                r[name] = e
            out[k["config"]] = r
            continue
        ci = k["chain_index"]
        probs = k["problems"]
        n_prob = len(ci) if ci is not None else m.n_chains
        probs = list(range(n_prob)) if probs is None else probs
        kw = dict(chain_index=ci, state_offsets=k.get("state_offsets"),
                  n_threads=os.cpu_count() or 1)
        if k["problems"] is not None:
            kw["problems"] = probs
        t0 = time.perf_counter()
        ref = oracle.fd(m, st.q, st.qdot, st.tau, algo="cholesky", **kw)
        t1 = time.perf_counter()
        aba = oracle.fd(m, st.q, st.qdot, st.tau, algo="aba", **kw)
        t2 = time.perf_counter()
        # the CPU baseline of this configuration: the oracle's two routes on the
        # sampled problems (OpenMP across problems)
        cpu_cfg = {"kind": "oracle", "cores": kw["n_threads"], "problems": len(probs),
                   "cholesky_solves_per_s": len(probs) / max(t1 - t0, 1e-9),
                   "aba_solves_per_s": len(probs) / max(t2 - t1, 1e-9),
                   "sample": f"{len(probs)} of {n_prob} problems, FP64"}
        f32 = lambda a: a.astype(np.float32).astype(np.float64)
        ref32 = None
        if any(not name.endswith(("fp64",)) and "mixed" in name for name in k["outs"]):
            ref32 = oracle.fd(m, f32(st.q), f32(st.qdot), f32(st.tau), algo="cholesky", **kw)
        offs = m.offsets if ci is None else np.asarray(k["state_offsets"])

        def err(x, rf=ref):
            e = 0.0
            for p in probs:
                a, b = int(offs[p]), int(offs[p + 1])
                e = max(e, float(np.abs(x[a:b] - rf[a:b]).max() / max(np.abs(rf[a:b]).max(), 1.0)))
            return e
        r = {"sampled_problems": len(probs), "oracle_aba_floor": err(aba), "cpu_oracle": cpu_cfg}
        for name, x in k["outs"].items():
            r[name] = err(x)
            if ref32 is not None and "mixed" in name:
                r[name + "_vs_states_rounded_to_fp32"] = err(x, ref32)
        out[k["config"]] = r
    return out


def reference_arm(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    model = synth.random_chains([args.links] * args.chains, seed=0)
    st = synth.random_states(model.n_links_total, seed=1)
    import oracle
    threads = os.cpu_count() or 1
    sample = 512
    L = sample * args.links
    sub = synth.ChainModel(model.axes[:L], model.frames[:L], model.inertias[:L],
                           model.offsets[:sample + 1].copy(), model.gravity)
    algos = {"abia": "aba", "jsiia": "cholesky", "cfa": "cfa"}
    for _ in range(args.warmup):
        oracle.fd(sub, st.q[:L], st.qdot[:L], st.tau[:L], algo="cfa", n_threads=threads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for a in ALGOS:
            oracle.fd(sub, st.q[:L], st.qdot[:L], st.tau[:L], algo=algos[a], n_threads=threads)
    el = time.perf_counter() - t0
    val = 3 * sample * args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "FD solves/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "chains": args.chains, "links": args.links,
                       "step": f"ABIA+JSIIA+CFA on a bounded sample of {sample} chains"},
            "cpu_baseline": {"value": val, "unit": "FD solves/s", "cores": threads,
                             "kind": "oracle",
                             "sample": f"{sample} of {args.chains} chains per step"},
            "e2e": {"value": val, "unit": "FD solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    from paper_1609_06779_gb300 import fd

    if not args.no_peak:
        measure_peak(fd, local)

    # weak scaling: every rank solves its own 65 536-chain batch (no data exchange)
    model = synth.random_chains([args.links] * args.chains, seed=rank)
    st = synth.random_states(model.n_links_total, seed=1000 + rank)
    cs = fd.ChainSet(model, device=local)
    batch = fd.Batch(cs)
    t = lambda a, dt: torch.tensor(a, dtype=dt, device=dev)
    q, qd, tau = (t(x, torch.float64) for x in (st.q, st.qdot, st.tau))
    out = {a: torch.empty_like(q) for a in ALGOS}
    teams = {}
    forced = fixed_teams(args.teams)
    for a in ALGOS:  # schedule per algorithm, chosen by timing (untimed here)
        teams[a] = forced.get(a) or fd.autotune(batch, q, qd, tau, algo=a, prec="fp64")
    torch.cuda.empty_cache()
    ws = {a: fd.workspace(batch, a, "fp64", teams[a], dev) for a in ALGOS}
    stream = torch.cuda.current_stream(dev)

    def step(evs=None):
        for k, a in enumerate(ALGOS):
            if evs is not None:
                evs[k].record(stream)
            fd.solve(batch, q, qd, tau, algo=a, prec="fp64", team=teams[a], out=out[a],
                     ws=ws[a], stream=stream)
        if evs is not None:
            evs[3].record(stream)

    for _ in range(max(args.warmup, 1)):
        step()
    torch.cuda.synchronize()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    clk = Clocks(os.path.join(tempfile.gettempdir(), f"fd_bench_clocks_{os.getpid()}.csv"), local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with clk:
        time.sleep(0.3)
        t_begin = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_begin.record(stream)
        for s in range(args.steps):
            step(evs[s])
        t_end.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    total_ms = t_begin.elapsed_time(t_end)
    per_algo_ms = {a: float(np.mean([evs[s][k].elapsed_time(evs[s][k + 1])
                                     for s in range(args.steps)])) for k, a in enumerate(ALGOS)}
    total_ms = fdist.max_over_ranks(total_ms, dev)
    solves = 3 * args.chains * world * args.steps
    value = solves / (total_ms / 1e3)

    # per-algorithm roofline (FP64 pipe: the kernels are ALU bound)
    lengths = [args.links] * args.chains
    rl = {}
    for a in ALGOS:
        fl = roofline.flops(a, lengths)
        ach = fl / (per_algo_ms[a] / 1e3) / 1e12
        rl[a] = {"ms": per_algo_ms[a], "tflops": ach, "frac": ach / FP64_PEAK_TFLOPS,
                 "solves_per_s": args.chains / (per_algo_ms[a] / 1e3)}
    dom = max(ALGOS, key=lambda a: per_algo_ms[a])
    tr = traffic_record(f"{dom}_kernel", teams[dom])
    traffic = None
    if tr is not None:
        # DRAM bytes of one launch: the capture's bytes per link x this launch's links
        traffic = tr["bytes_per_link"] * args.chains * args.links
    hbm_peak = measured_hbm_gbs()
    alg_bytes = roofline.bytes_per_link("fp64") * args.chains * args.links
    hbm_gbs = alg_bytes / (per_algo_ms[dom] / 1e3) / 1e9
    roof = {"bound": "alu", "achieved": rl[dom]["tflops"], "peak": FP64_PEAK_TFLOPS,
            "unit": "TFLOP/s", "frac": rl[dom]["frac"], "traffic": traffic,
            "kernel": f"{dom}_kernel, team {teams[dom]}, FP64",
            "peak_source": PEAK_INFO,
            "algorithmic_flops_per_launch": roofline.flops(dom, lengths),
            "algorithmic_bytes_per_launch": alg_bytes,
            "hbm": {"achieved_gbs": hbm_gbs, "peak_gbs": hbm_peak,
                    "frac": (hbm_gbs / hbm_peak) if hbm_peak else None,
                    "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured copy)"}}

    # the first chains' results of every path, for the accuracy check of the CPU leg
    # every chain's FP64 result, the first 4 096 chains' FP32 / mixed results
    n_acc = min(args.chains, 4096) * args.links
    acc_outs = {f"{a}_fp64": out[a].cpu() for a in ALGOS}

    # CFA with block cyclic reduction in place of OEE (context; not part of the step)
    variants = {}
    if rank == 0 and not args.no_variants:
        for var in ("cfa_cr", "cfa_hybrid"):
            tcr = forced.get(var) or fd.autotune(batch, q, qd, tau, algo=var, prec="fp64")
            wcr = fd.workspace(batch, var, "fp64", tcr, dev)
            ocr = torch.empty_like(q)
            ms = _time_ms(lambda: fd.solve(batch, q, qd, tau, algo=var, team=tcr, out=ocr,
                                           ws=wcr), reps=5, warm=2)
            fl = roofline.flops(var, lengths)
            acc_outs[f"{var}_fp64"] = ocr.cpu()
            variants[f"{var}_fp64"] = {"team": tcr, "ms": ms,
                                       "solves_per_s": args.chains / (ms * 1e-3),
                                       "tflops": fl / (ms * 1e-3) / 1e12,
                                       "frac": fl / (ms * 1e-3) / 1e12 / FP64_PEAK_TFLOPS}
            del wcr, ocr
        # inverse dynamics alone (fd_inverse_dynamics, the scans of Eq. 2a-2d) and the
        # adjoint (FD and M^-1 w in one elimination, then the reverse sweep) of CFA
        for team in (8,):
            wid = fd.workspace(batch, None, "fp64", team, dev)
            oid = torch.empty_like(q)
            ms = _time_ms(lambda: fd.inverse_dynamics(batch, q, qd, out["cfa"], team=team,
                                                      out=oid, ws=wid), reps=5, warm=2)
            fl = roofline.flops("id", lengths)
            variants["inverse_dynamics_fp64"] = {"team": team, "ms": ms,
                                                 "solves_per_s": args.chains / (ms * 1e-3),
                                                 "tflops": fl / (ms * 1e-3) / 1e12}
            del wid, oid
        wb = torch.randn_like(q)
        ms = _time_ms(lambda: fd.adjoint(batch, q, qd, tau, wb, algo="cfa", team=teams["cfa"],
                                         masses=False), reps=3, warm=1)
        variants["adjoint_cfa_fp64"] = {"team": teams["cfa"], "ms": ms,
                                        "solves_per_s": args.chains / (ms * 1e-3)}
        del wb
        # the step's three launches on three streams forked from and joined to the
        # launching stream: the GPU fills one kernel's tail with the others' blocks
        side = [torch.cuda.Stream(dev) for _ in ALGOS]

        def step3():
            fork = torch.cuda.Event()
            fork.record(stream)
            for s, a in zip(side, ALGOS):
                s.wait_event(fork)
                fd.solve(batch, q, qd, tau, algo=a, prec="fp64", team=teams[a], out=out[a],
                         ws=ws[a], stream=s)
            for s in side:
                join = torch.cuda.Event()
                join.record(s)
                stream.wait_event(join)

        ms = _time_ms(step3, reps=5, warm=2)
        torch.cuda.synchronize()
        same3 = all(torch.equal(out[a].cpu(), acc_outs[f"{a}_fp64"]) for a in ALGOS)
        variants["step_three_streams_fp64"] = {"ms": ms,
                                               "solves_per_s": 3 * args.chains / (ms * 1e-3),
                                               "results_equal_device_step": same3}
    # FP32 and mixed variants of each algorithm (context; not part of the step)
    if rank == 0 and not args.no_variants:
        q32, qd32, tau32 = (x.float() for x in (q, qd, tau))
        for prec in ("fp32", "mixed"):
            for a in ALGOS:
                tv = forced.get(a, 0)
                if not tv:
                    fd.autotune(batch, q32, qd32, tau32, algo=a, prec=prec)
                w = fd.workspace(batch, a, prec, tv, dev)
                o = torch.empty_like(q32)
                for _ in range(2):
                    fd.solve(batch, q32, qd32, tau32, algo=a, prec=prec, team=tv,
                             out=o, ws=w)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(3):
                    fd.solve(batch, q32, qd32, tau32, algo=a, prec=prec, team=tv,
                             out=o, ws=w)
                e1.record(stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / 3
                variants[f"{a}_{prec}"] = {"ms": ms, "solves_per_s": args.chains / (ms / 1e3)}
                acc_outs[f"{a}_{prec}"] = o[:n_acc].cpu()
                del w
        # CFA on the block-Jacobi projection (fd_solve_cfa_projected: W_i = Wc_i
        # L_i^{-T}, the paper's open choice of W in Eq. cfa-eq1): the same qdd,
        # another elimination's rounding
        for prec, (qq, qqd, qtau) in (("fp64", (q, qd, tau)), ("fp32", (q32, qd32, tau32))):
            tv = forced.get("cfa", 0)
            w = fd.workspace(batch, "cfa", prec, tv, dev)
            o = torch.empty_like(qq)
            ms = _time_ms(lambda: fd.solve_cfa_projected(batch, qq, qqd, qtau,
                                                         projection="block_jacobi", prec=prec,
                                                         team=tv, out=o, ws=w), reps=3, warm=2)
            variants[f"cfa_block_jacobi_{prec}"] = {"ms": ms,
                                                    "solves_per_s": args.chains / (ms / 1e3)}
            acc_outs[f"cfa_block_jacobi_{prec}"] = o.cpu() if prec == "fp64" else o[:n_acc].cpu()
            del w, o

    # end to end through the C ABI with host buffers (pinned), copies timed: every
    # step copies its inputs host -> device and its three results device -> host.
    # The copies run on their own streams beside the solves (pipelined: step s+1's
    # inputs go up into the other of two device buffers while step s solves, and
    # each result comes down while the next algorithm runs).
    e2e = None
    if not args.no_e2e:
        hq, hqd, htau = (x.cpu().pin_memory() for x in (q, qd, tau))
        hout = {a: torch.empty(q.shape, dtype=torch.float64).pin_memory() for a in ALGOS}
        dbuf = [tuple(torch.empty_like(q) for _ in range(3)) for _ in range(2)]
        s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)

        def e2e_run(k):
            ev_in, ev_free = [None, None], [None, None]
            ev_out = {a: None for a in ALGOS}

            def h2d(j):
                if ev_free[j] is not None:      # the step that last read buffer j has solved
                    s_in.wait_event(ev_free[j])
                with torch.cuda.stream(s_in):
                    for d, h in zip(dbuf[j], (hq, hqd, htau)):
                        d.copy_(h, non_blocking=True)
                ev_in[j] = torch.cuda.Event()
                ev_in[j].record(s_in)

            h2d(0)
            for st_i in range(k):
                j = st_i % 2
                if st_i + 1 < k:
                    h2d(1 - j)
                stream.wait_event(ev_in[j])
                for a in ALGOS:
                    if ev_out[a] is not None:   # the previous step's result has come down
                        stream.wait_event(ev_out[a])
                    fd.solve(batch, *dbuf[j], algo=a, prec="fp64", team=teams[a], out=out[a],
                             ws=ws[a], stream=stream)
                    done = torch.cuda.Event()
                    done.record(stream)
                    s_out.wait_event(done)
                    with torch.cuda.stream(s_out):
                        hout[a].copy_(out[a], non_blocking=True)
                    ev_out[a] = torch.cuda.Event()
                    ev_out[a].record(s_out)
                ev_free[j] = torch.cuda.Event()
                ev_free[j].record(stream)
            stream.wait_stream(s_out)

        e2e_run(2)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ksteps = max(1, min(args.steps, 5))
        e2e_run(ksteps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        ms = fdist.max_over_ranks(ms, dev)
        nb = q.numel() * 8
        # the results that came down equal the device-timed step's, bit for bit
        same = all(torch.equal(hout[a], acc_outs[f"{a}_fp64"]) for a in ALGOS)
        e2e = {"value": 3 * args.chains * world * ksteps / (ms / 1e3), "unit": "FD solves/s",
               "h2d_bytes_per_step": 3 * nb, "d2h_bytes_per_step": 3 * nb,
               "steps": ksteps, "copies": "own streams, pipelined with the solves",
               "results_equal_device_step": same}

    del ws, out
    torch.cuda.empty_cache()
    extra = None
    keep = []
    if rank == 0 and not args.no_extra:
        extra = extra_configs(dev, keep)
        torch.cuda.empty_cache()
    serving = None
    if rank == 0 and not args.no_serve:
        serving = {"continuous": serve_bench(args.serve_seconds, args.serve_rate, False,
                                             device=local),
                   "per_size_baseline": serve_bench(args.serve_seconds, args.serve_rate, True,
                                                    device=local)}

    cpu = acc = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_oracle(model, st, args.chains)
        acc = accuracy(model, st, acc_outs)
        if keep:
            acc["configs"] = config_accuracy(keep)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "FD solves/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": WORKLOAD, "chains_per_gpu": args.chains,
                           "links": args.links, "step": "ABIA + JSIIA + CFA, FP64, one launch each",
                           "team": teams,
                           "l2": "inputs larger than L2 (FP64 model arena 940 MB), no flush",
                           "parallelism": f"replicas x{world}, chains partitioned, no exchange"},
                "per_algo": rl, "variants": variants,
                "roofline": roof, "cpu_baseline": cpu, "accuracy": acc, "e2e": e2e,
                "serving": serving,
                "configs": extra,
                "gpu_launches": 3 * args.steps, "clocks": clk.summary()}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
