#!/usr/bin/env python3
"""Benchmark of the embedding hot path on GB300.

One step = the whole hot path on one seeded synthetic manifold graph: the operator build
(two-hop CSR assembly, Q, eps = lambda_2(Q) by LOBPCG, mu, A, B; Sec. 4) and the LOBPCG
solve for the first K generalized eigenpairs of (A, B) (Sec. 4.3).  The graph (the kNN
construction of Sec. 5.1, seeded points on a 3-D swiss roll) is input preparation and is
not timed.

Default workload: N = 200,000 points on a swiss roll, symmetric 10-NN graph with Gaussian
weights, K = 8, relative-residual tolerance 1e-5 (||A x - lambda B x||_{B^-1} <= 1e-5 |lambda|
||x||_B per pair), FP32 blocks.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun each rank embeds its own graph (seed + rank,
same size): independent problems, no collective on the data path ("scaling": "weak").
The reference arm (--impl reference) times the CPU oracle on a bounded sample of the same
workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

UNIT = "node-embeddings/s"


def metric(a):
    tol = ("%g" % a.tol).replace("e-0", "e-")
    return f"node-embeddings/s (K={a.K} generalized eigenvectors per node, relative residual <= {tol})"


def accuracy_note(a):
    """Where the accuracy of this workload's results is checked."""
    w = (a.shape, a.n, a.knn, a.K, a.seed)
    if w == ("swiss_roll", 200_000, 10, 8, 2) and a.precision in ("fp32", "bf16"):
        return ("eigenvalues within 1.9e-6 relative and eigenvectors within 1.6e-6 rad (FP32; BF16 form 2.9e-6, "
                "3.1e-5 rad) of the oracle's machine-precision pairs on this workload (tests/test_gpu_fullsize.py)")
    if w == ("sphere", 2_000_000, 10, 16, 3) and a.precision == "fp32":
        return ("pairs checked by properties at this size (tests/test_gpu_sphere_2m.py): backward error <= 1e-6 "
                "against the oracle's FP64 A and b, V^T B V = I, the sphere's 1-3-5-7 eigenvalue groups, eps "
                "within the Courant-Fischer bracket")
    if w[:2] == ("square", 1000) and a.precision == "fp64":
        return "dense FP64 oracle parity on 1k-node graphs (tests/test_gpu_embed.py)"
    return "not measured at this size"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--warmup-seconds", type=float, default=2.0,
                   help="keep warming up (untimed) until at least this much wall time has passed")
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=200_000)
    p.add_argument("--shape", default="swiss_roll")
    p.add_argument("--knn", type=int, default=10)
    p.add_argument("--K", type=int, default=8)
    p.add_argument("--tol", type=float, default=1e-5)
    p.add_argument("--precision", default="fp32")
    p.add_argument("--seed", type=int, default=2)
    p.add_argument("--cpu-sample-n", type=int, default=5_000)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--serve-requests", type=int, default=32)
    p.add_argument("--no-serving", action="store_true")
    p.add_argument("--serve-budget-gb", type=float, default=16.0,
                   help="HBM budget of the serving context (admission by footprint)")
    p.add_argument("--batch-graphs", type=int, default=512)
    p.add_argument("--no-extras", action="store_true", help="skip the kNN, k-means and betweenness lines")
    p.add_argument("--no-batch", action="store_true")
    p.add_argument("--no-sphere-2m", action="store_true", help="skip the 2M-node sphere (K = 16) line")
    p.add_argument("--autotune", type=int, default=1, choices=[0, 1],
                   help="1: the Chebyshev step's autotuner (default); 0: its fixed rule, for comparison")
    p.add_argument("--autotune-cache", default=None,
                   help="JSON cache of the Chebyshev step's tuned configurations shared by the bench's contexts "
                        "(default: a new temporary file); read first if it exists")
    p.add_argument("--batch-workers", type=int, default=8, help="host threads of mge_build_graph_ops_batch")
    p.add_argument("--oracle-step-only", action="store_true", help=argparse.SUPPRESS)
    return p.parse_args()


def workload(a, n=None):
    return {"workload": f"{a.shape} N={n or a.n} {a.knn}-NN K={a.K} tol={a.tol:g} {a.precision} blocks",
            "shape": a.shape, "n": n or a.n, "knn": a.knn, "K": a.K, "tol": a.tol,
            "precision": a.precision, "seed": a.seed}


# ---------------------------------------------------------------------------------------
# distributed plumbing (barrier and max-over-ranks only; no data-path collective)
# ---------------------------------------------------------------------------------------
class Dist:
    def __init__(self, backend):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch.distributed as dist
            os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
            dist.init_process_group(backend=backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            if self.pg.get_backend() == "nccl":
                import torch
                self.pg.barrier(device_ids=[torch.cuda.current_device()])
            else:
                self.pg.barrier()

    def max(self, x: float) -> float:
        if not self.pg:
            return x
        import torch
        dev = "cuda" if self.pg.get_backend() == "nccl" else "cpu"
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


# ---------------------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        fd, self.path = tempfile.mkstemp(prefix=f"mge_clocks_gpu{gpu}_", suffix=".csv")
        os.close(fd)

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() in ("active", "1"):
                    reasons.add(nm)
        if not sm:
            return None
        busy = [s for s in sm if mx is None or s > 0.5 * mx] or sm
        return {"sm_mhz": statistics.median(busy), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------------------
def spmm_traffic_per_launch():
    """DRAM bytes per SpMM launch from the committed ncu summary, if the kernel source it was
    taken from is unchanged; otherwise null."""
    path = os.path.join(ROOT, "profiles", "spmm_traffic.json")
    if not os.path.exists(path):
        return None
    try:
        d = json.load(open(path))
        src = b"".join(open(os.path.join(ROOT, "paper_2112_07862_gb300", "csrc", f), "rb").read()
                       for f in ("lobpcg.cu", "cheb.cu"))
        if d.get("source_sha256") != hashlib.sha256(src).hexdigest():
            return None
        return d.get("dram_bytes_per_launch")
    except Exception:
        return None


def run_ours(a, dist):
    import numpy as np
    import torch

    import manifold_graphs as mg
    from paper_2112_07862_gb300 import mge

    torch.cuda.set_device(dist.local)
    g = mg.manifold_graph(a.shape, a.n, a.knn, a.seed + dist.rank)
    ctx = mge.Context(dist.local)
    # the Chebyshev step's configurations tuned during the warm-up, reported with the line
    tune_path = tune_cache(a)
    mge.mge_ctx_set_autotune(ctx.h, a.autotune, tune_path)
    stream = torch.cuda.current_stream()
    sptr = stream.cuda_stream
    # device-resident inputs for the kernel-level number
    rp_d = torch.from_numpy(g.row_ptr).cuda()
    col_d = torch.from_numpy(g.col).cuda()
    w_d = torch.from_numpy(g.w).cuda()
    V_d = torch.empty((a.K, g.n), dtype=torch.float64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")   # > L2 (129 MB)
    oo = mge.ops_opts(a.precision, stream=sptr)
    eo = mge.embed_opts(a.precision, v_on_device=True, stream=sptr)
    status = {"build": None, "embed": None, "m": None}
    phases = {"build_ms": [], "embed_ms": [], "eps_iters": []}

    def step():
        flush.zero_()
        h, s = mge.mge_build_graph_ops(ctx.h, g.n, rp_d, col_d, w_d, True, oo)
        lam, V, info, s2 = mge.mge_embed(ctx.h, h, a.K, a.tol, eo, V_d)
        oi = mge.mge_ops_info(h)
        phases["build_ms"].append(oi.build_ms)
        phases["eps_iters"].append(oi.eps_iters)
        phases["embed_ms"].append(info.solve_ms)
        mge.mge_ops_destroy(h)
        status["build"], status["embed"], status["m"] = s, s2, info.m
        return lam, info

    # at least W untimed steps, and at least warmup_seconds of them: the first seconds of a fresh
    # process and GPU run slower (measured: 2.1M node-embeddings/s for the first bench process
    # of a call against 3.1M for a later one, at the same clocks)
    t_w = time.perf_counter()
    warm_run = 0
    while warm_run < a.warmup or time.perf_counter() - t_w < a.warmup_seconds:
        step()
        warm_run += 1
    torch.cuda.synchronize()
    for v in phases.values():
        v.clear()
    clocks = ClockSampler(dist.local)
    clocks.start()
    dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    iters = []
    for _ in range(a.steps):
        lam, info = step()
        iters.append(info.iters)
    e1.record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    # per-launch SpMM times for the roofline: one more step with the library's event timing
    # on (outside the timed region: the events around every SpMM launch cost time)
    mge.mge_ctx_reset_stats(ctx.h)
    mge.mge_ctx_set_timing(ctx.h, True)
    step()
    torch.cuda.synchronize()
    mge.mge_ctx_set_timing(ctx.h, False)
    st = mge.mge_ctx_stats(ctx.h)
    ms_max = dist.max(ms)
    per_step = ms_max / a.steps
    value = dist.world * g.n * a.steps / (ms_max / 1e3)

    # end to end through the public API with host buffers: H2D of W inside the call, V back
    e2e = None
    if not a.no_e2e:
        rp_h = torch.from_numpy(g.row_ptr).pin_memory()
        col_h = torch.from_numpy(g.col).pin_memory()
        w_h = torch.from_numpy(g.w).pin_memory()
        V_h = torch.empty((a.K, g.n), dtype=torch.float64).pin_memory()
        oo_h = mge.ops_opts(a.precision, stream=sptr)
        eo_h = mge.embed_opts(a.precision, v_on_device=False, stream=sptr)

        def step_e2e():
            flush.zero_()
            h, s = mge.mge_build_graph_ops(ctx.h, g.n, rp_h.numpy(), col_h.numpy(), w_h.numpy(), False, oo_h)
            lam, V, info, s2 = mge.mge_embed(ctx.h, h, a.K, a.tol, eo_h, V_h.numpy())
            mge.mge_ops_destroy(h)
            return lam

        step_e2e()
        torch.cuda.synchronize()
        dist.barrier()
        t0 = time.perf_counter()
        for _ in range(a.steps):
            step_e2e()
        torch.cuda.synchronize()
        t_e2e = dist.max(time.perf_counter() - t0)
        e2e = {"value": dist.world * g.n * a.steps / t_e2e, "unit": UNIT,
               "h2d_bytes_per_step": int(g.row_ptr.nbytes + g.col.nbytes + g.w.nbytes),
               "d2h_bytes_per_step": int(V_h.numel() * 8 + a.K * 8),
               "ms_per_step": 1e3 * t_e2e / a.steps}

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = peaks.get("hbm_gbs")
    peak_src = "of measured"
    if not hbm:
        hbm, peak_src = 6800.0, "of fallback"
    achieved = (st.spmm_bytes / (st.spmm_ms / 1e3) / 1e9) if st.spmm_ms > 0 else None
    traffic = spmm_traffic_per_launch()
    # the SpMMs of both solves: k_cheb, the Chebyshev preconditioner steps (degree - 1 per
    # iteration, on L + eps I in the embedding and on Q in the eps solve), and k_spmm_w, the
    # operator product with the fused projection/normalisation of W (once per iteration);
    # achieved = algorithmic bytes of all timed launches / their summed event time
    roofline = {"kernel": "k_cheb (Chebyshev preconditioner steps) and k_spmm_w (A W_raw, fused projection)",
                "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": (achieved / hbm) if achieved else None, "peak_source": peak_src,
                "traffic": traffic, "launches_timed": st.spmm_launches,
                "avg_launch_us": 1e3 * st.spmm_ms / st.spmm_launches if st.spmm_launches else None,
                "algorithmic_bytes_per_launch": st.spmm_bytes / st.spmm_launches if st.spmm_launches else None}
    res = {
        "metric": metric(a), "value": value, "unit": UNIT, "n_gpus": dist.world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if a.precision == "fp32" else a.precision.replace("fp", "f"),
        "data": f"synthetic: seeded {a.shape.replace('_', '-')} points, exact symmetric kNN graph, Gaussian weights",
        "config": dict(workload(a), l2="flushed (256 MB write) before every step",
                       parallelism=f"replicas x{dist.world} (independent graphs, no collective)"),
        "gpu_launches": int(st.kernel_launches) * a.steps,
        "warmup_steps_run": warm_run,
        "lobpcg_iters_per_step": statistics.mean(iters),
        "lobpcg_block_m": status["m"],
        "phases": {"build_ms": statistics.mean(phases["build_ms"][:a.steps]),
                   "embed_ms": statistics.mean(phases["embed_ms"][:a.steps]),
                   "eps_iters": statistics.mean(phases["eps_iters"][:a.steps])},
        "status": {"build": status["build"], "embed": status["embed"]},
        "accuracy_note": accuracy_note(a),
        "roofline": roofline,
        "e2e": e2e,
        "clocks": clk,
        "autotune": _read_json(tune_path),
    }
    ctx.close()
    return res


# ---------------------------------------------------------------------------------------
# the batching form: many graphs of uneven size in one graph launch (mge_embed_batch)
# ---------------------------------------------------------------------------------------
def run_batch(a):
    """Graphs with N log-uniform in [2,000, 50,000], shape square / torus / swiss roll, k in
    {8, 10, 12}, K in {4, 8} (seed 4 + index), FP32 blocks, tol 1e-5.  The points are sampled
    on the host; their kNN graphs are built on the device (mge_knn_graph), the operators by
    mge_build_graph_ops_batch (concurrent builds on 8 host threads and streams; timed against
    one mge_build_graph_ops after another); then every embedding runs as a branch of ONE CUDA
    graph launch and, for comparison, one mge_embed after another.
    Embedding throughput = sum of N / device time of the launch(es)."""
    import numpy as np
    import torch

    import manifold_graphs as mg
    from paper_2112_07862_gb300 import mge

    rng = np.random.default_rng(4)
    shapes = ["square", "torus", "swiss_roll"]
    specs = []
    for i in range(a.batch_graphs):
        n = int(round(float(np.exp(rng.uniform(np.log(2_000), np.log(50_000))))))
        shape = shapes[int(rng.integers(3))]
        k = int(rng.choice([8, 10, 12]))
        K = int(rng.choice([4, 8]))
        specs.append((mg.sample_points(shape, n, 4 + i), k, K))
    nodes = sum(P.shape[0] for P, _, _ in specs)
    Ks = [K for _, _, K in specs]
    with mge.Context(0) as ctx:
        mge.mge_ctx_set_autotune(ctx.h, a.autotune, tune_cache(a))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        graphs = [mge.mge_knn_graph(ctx.h, P, k) for P, k, _ in specs]
        t_knn = time.perf_counter() - t0
        csr = []
        for g in graphs:
            n, _, _ = mge.mge_graph_info(g)
            rp, col, w = mge.mge_graph_csr(g)
            csr.append((n, rp, col, w))
        t0 = time.perf_counter()
        for n, rp, col, w in csr:
            mge.mge_ops_destroy(mge.mge_build_graph_ops(ctx.h, n, rp, col, w, True, mge.ops_opts("fp32"))[0])
        t_build_seq = time.perf_counter() - t0
        t0 = time.perf_counter()
        ops, _, _ = mge.mge_build_graph_ops_batch(ctx.h, csr, True, mge.ops_opts("fp32"), workers=a.batch_workers)
        t_build = time.perf_counter() - t0
        for g in graphs:
            mge.mge_graph_destroy(g)
        eo = mge.embed_opts("fp32")
        mge.mge_embed_batch(ctx.h, ops, Ks, a.tol, eo)            # warm-up (allocations, instantiation)
        t0 = time.perf_counter()
        lams, Vs, infos, s = mge.mge_embed_batch(ctx.h, ops, Ks, a.tol, eo)
        t_batch = time.perf_counter() - t0
        dev_batch = infos[0].solve_ms
        t0 = time.perf_counter()
        dev_seq = 0.0
        for o, K in zip(ops, Ks):
            dev_seq += mge.mge_embed(ctx.h, o, K, a.tol, eo)[2].solve_ms
        t_seq = time.perf_counter() - t0
        for o in ops:
            mge.mge_ops_destroy(o)
    iters = [i.iters for i in infos]
    return {"graphs": len(specs), "nodes": int(nodes), "status": int(s),
            "converged": int(sum(1 for i in infos if i.status == 0)),
            "value": nodes / (dev_batch / 1e3), "unit": UNIT,
            "batch_launch_ms": dev_batch, "batch_call_ms": 1e3 * t_batch,
            "one_by_one_device_ms": dev_seq, "one_by_one_call_ms": 1e3 * t_seq,
            "one_by_one_value": nodes / (dev_seq / 1e3),
            "knn_ms": 1e3 * t_knn,
            "build_ms_batch": 1e3 * t_build, "build_ms_one_by_one": 1e3 * t_build_seq,
            "with_build_value": nodes / (t_knn + t_build + t_batch),
            "iters_min_max": [min(iters), max(iters)],
            "workload": f"{len(specs)} graphs, N log-uniform in [2000, 50000] (seed 4 + index), square/torus/"
                        "swiss roll, k in {8,10,12}, K in {4,8}, FP32 blocks, relative residual 1e-5; value = "
                        "sum N / device time of the one batch launch (embedding only); with_build_value = sum N / "
                        "(wall time of the kNN graphs on the device + mge_build_graph_ops_batch (8 host threads "
                        "and streams) + the batch embedding call), host points in, host V out"}


# ---------------------------------------------------------------------------------------
# the serving form: Poisson arrivals through mge_submit / mge_poll
# ---------------------------------------------------------------------------------------
def run_serving(a):
    """Requests of uneven size arrive as a Poisson stream (200 req/s, seed 5): N log-uniform
    in [1,000, 500,000], shape square / sphere / swiss roll, 10-NN, K in {2, 4, 8, 16},
    FP32 or BF16 (seeded choice), relative residual 1e-5.  Each request carries its points:
    the library builds the kNN graph, the operators and the embedding on the device.  Requests
    are submitted at their arrival times and the library's slots admit and run them
    concurrently.  Latency is the library's submit-to-completion time."""
    import numpy as np

    import manifold_graphs as mg
    from paper_2112_07862_gb300 import mge

    rng = np.random.default_rng(5)
    shapes = ["square", "sphere", "swiss_roll"]
    reqs = []
    for i in range(a.serve_requests):
        n = int(round(float(np.exp(rng.uniform(np.log(1_000), np.log(500_000))))))
        shape = shapes[int(rng.integers(3))]
        K = int(rng.choice([2, 4, 8, 16]))
        # FP32 blocks: the BF16 form is slower on this path (no faster per Chebyshev step, more
        # iterations at its capped preconditioner degree); its place in a mixed stream is
        # covered by tests/test_gpu_serving.py
        prec = mge.MGE_FP32
        reqs.append((np.ascontiguousarray(mg.sample_points(shape, n, 500 + i)), K, prec))
    arrivals = np.cumsum(rng.exponential(1.0 / 200.0, len(reqs)))

    def request(P, K, prec):
        r = mge.mge_request()
        r.n, r.points, r.dim, r.knn = P.shape[0], P.ctypes.data, P.shape[1], 10
        r.K, r.tol, r.precision, r.guard, r.maxiter, r.seed = K, a.tol, prec, 0, 0, 0
        return r

    import threading
    budget = int(a.serve_budget_gb * (1 << 30))
    with mge.Context(0, budget) as ctx:
        mge.mge_ctx_set_autotune(ctx.h, 2 * a.autotune, tune_cache(a))
        # one small request first, so that the slots and their streams exist
        P0 = np.ascontiguousarray(mg.sample_points("square", 1_000, 499))
        t = mge.mge_submit(ctx.h, request(P0, 2, mge.MGE_FP32))
        mge.mge_poll(ctx.h, t, -1)
        mge.mge_release(ctx.h, t)
        # the context's device bytes while the stream runs (admission keeps them under the budget)
        peak = {"bytes": 0}
        done = threading.Event()

        def sample():
            while not done.is_set():
                peak["bytes"] = max(peak["bytes"], int(mge.mge_ctx_stats(ctx.h).hbm_in_use))
                time.sleep(0.002)
        sampler = threading.Thread(target=sample, daemon=True)
        sampler.start()
        tickets = []
        t0 = time.perf_counter()
        for (P, K, prec), ta in zip(reqs, arrivals):
            dt = t0 + ta - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            tickets.append(mge.mge_submit(ctx.h, request(P, K, prec)))
        lat, queue, ok, statuses = [], [], 0, {}
        for t in tickets:
            s, r = mge.mge_poll(ctx.h, t, -1)
            if s == mge.MGE_OK and r.status == mge.MGE_OK:
                ok += 1
            key = mge.mge_strerror(r.status if s == mge.MGE_OK else s)
            statuses[key] = statuses.get(key, 0) + 1
            lat.append(r.latency_ms)
            queue.append(r.queue_ms)
            mge.mge_release(ctx.h, t)
        wall = time.perf_counter() - t0
        done.set()
        sampler.join()
    nodes = sum(P.shape[0] for P, _, _ in reqs)
    return {"requests": len(reqs), "bf16_requests": int(sum(1 for _, _, p in reqs if p == mge.MGE_BF16)), "converged": ok, "statuses": statuses, "offered_req_per_s": 200.0,
            "served_req_per_s": len(reqs) / wall, "value": nodes / wall, "unit": UNIT,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "queue_p50_ms": float(np.percentile(queue, 50)), "queue_p99_ms": float(np.percentile(queue, 99)),
            "nodes": int(nodes), "wall_s": wall,
            "workload": "Poisson 200 req/s (seed 5), N log-uniform in [1000, 500000], square/sphere/swiss "
                        "roll, 10-NN, K in {2,4,8,16}, FP32 blocks, relative residual 1e-5; each request "
                        "carries its points (kNN graph, operators and embedding on the device); latency = submit "
                        "to completion (host clock), host points in, host V out",
            "slots": int(os.environ.get("MGE_SERVE_SLOTS", "4")),
            "hbm_budget_bytes": budget, "hbm_peak_bytes": peak["bytes"]}


# ---------------------------------------------------------------------------------------
# the steps around the path: kNN graph from points, k-means of the embedding, VBC
# ---------------------------------------------------------------------------------------
def _event_ms(fn, reps=3):
    """Best device time of fn() over reps calls (CUDA events on torch's current stream, which
    fn's library calls are handed), after one untimed call."""
    import torch
    fn()
    best = None
    for _ in range(reps):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1)
        best = t if best is None else min(best, t)
    return best


def tune_cache(a):
    """One autotuning cache for every context of this run: shapes tuned in the warm-up are not
    tuned again later (the serving context only reads it, so that no tuning runs among its
    concurrent requests)."""
    if not a.autotune_cache:
        a.autotune_cache = os.path.join(tempfile.mkdtemp(prefix="mge_tune_"), "tune.json")
    return a.autotune_cache


def _read_json(path):
    try:
        return json.load(open(path))
    except Exception:
        return None


def run_sphere_2m(a):
    """The precision-form workload: 2,000,000 points uniform on the unit sphere (seed 3), exact
    10-NN graph built on the device from the points, operators + K = 16 embedding in FP32
    blocks to relative residual 1e-5.  Two timed steps after one warm-up, L2 flushed before
    each; one more step with the library's per-launch event timing gives the SpMM roofline."""
    import numpy as np
    import torch

    import manifold_graphs as mg
    from paper_2112_07862_gb300 import mge

    n, k, K, tol, seed = 2_000_000, 10, 16, 1e-5, 3
    stream = torch.cuda.current_stream()
    sptr = stream.cuda_stream
    tune_path = tune_cache(a)
    with mge.Context(0) as ctx:
        mge.mge_ctx_set_autotune(ctx.h, a.autotune, tune_path)
        P = torch.from_numpy(np.ascontiguousarray(mg.sample_points("sphere", n, seed))).cuda()
        g = mge.mge_knn_graph(ctx.h, P, k, stream=sptr)
        rp, col, w = mge.mge_graph_csr(g)
        V = torch.empty((K, n), dtype=torch.float64, device="cuda")
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
        oo = mge.ops_opts("fp32", stream=sptr)
        eo = mge.embed_opts("fp32", v_on_device=True, stream=sptr)
        rec = {}

        def step():
            flush.zero_()
            h, s = mge.mge_build_graph_ops(ctx.h, n, rp, col, w, True, oo)
            lam, _, info, s2 = mge.mge_embed(ctx.h, h, K, tol, eo, V)
            oi = mge.mge_ops_info(h)
            mge.mge_ops_destroy(h)
            rec.update(build=s, embed=s2, iters=info.iters, eps_iters=oi.eps_iters, build_ms=oi.build_ms,
                       embed_ms=info.solve_ms, rr64_from=info.rr_fp64_from)

        step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        steps = 2
        e0.record(stream)
        for _ in range(steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        mge.mge_ctx_reset_stats(ctx.h)
        mge.mge_ctx_set_timing(ctx.h, True)
        step()
        torch.cuda.synchronize()
        mge.mge_ctx_set_timing(ctx.h, False)
        st = mge.mge_ctx_stats(ctx.h)
        mge.mge_graph_destroy(g)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = peaks.get("hbm_gbs") or 6800.0
    achieved = st.spmm_bytes / (st.spmm_ms / 1e3) / 1e9 if st.spmm_ms > 0 else None
    return {"workload": "sphere N=2000000 10-NN (device kNN from the points) K=16 tol=1e-5 fp32 blocks, build + embed",
            "value": n / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "steps": steps, "warmup": 1,
            "status": {"build": rec["build"], "embed": rec["embed"]}, "lobpcg_iters": rec["iters"],
            "eps_iters": rec["eps_iters"], "build_ms": rec["build_ms"], "embed_ms": rec["embed_ms"],
            "rr_fp64_from": rec["rr64_from"], "l2": "flushed (256 MB write) before every step",
            "roofline": {"kernel": "k_cheb and k_spmm_w (working set above L2)", "bound": "hbm", "achieved": achieved,
                         "peak": hbm, "unit": "GB/s", "frac": achieved / hbm if achieved else None,
                         "launches_timed": int(st.spmm_launches),
                         "avg_launch_us": 1e3 * st.spmm_ms / st.spmm_launches if st.spmm_launches else None},
            "accuracy_note": accuracy_note(argparse.Namespace(shape="sphere", n=n, knn=k, K=K, seed=seed,
                                                              precision="fp32")),
            "autotune": {k: v for k, v in (_read_json(tune_path) or {}).items() if "/n2^20/" in k}}


def run_extras(a):
    import numpy as np
    import torch

    import manifold_graphs as mg
    from paper_2112_07862_gb300 import mge

    out = {}
    sptr = torch.cuda.current_stream().cuda_stream
    with mge.Context(0) as ctx:
        # kNN graph of the workload's points (device points in, device CSR out)
        P = mg.sample_points(a.shape, a.n, a.seed)
        Pd = torch.from_numpy(np.ascontiguousarray(P)).cuda()
        torch.cuda.synchronize()
        holder = {}

        def knn():
            if "g" in holder:
                mge.mge_graph_destroy(holder.pop("g"))
            holder["g"] = mge.mge_knn_graph(ctx.h, Pd, a.knn, stream=sptr)
        ms = _event_ms(knn)
        n, nnz, sigma = mge.mge_graph_info(holder["g"])
        out["knn"] = {"workload": f"{a.shape} N={a.n} points (dim {P.shape[1]}), exact {a.knn}-NN, union, "
                                  "Gaussian weights; device points in, device CSR out",
                      "ms": ms, "value": a.n / (ms / 1e3), "unit": "points/s", "nnz": int(nnz),
                      "launches_per_call": "13 kernels (bbox, 2 binning passes, scan, scatter, query, sigma, "
                                           "symmetrisation, weights)"}
        # k-means (C = 16, at most 50 steps) of that graph's embedding
        rp, col, w = mge.mge_graph_csr(holder["g"])
        h, s = mge.mge_build_graph_ops(ctx.h, n, rp, col, w, True, mge.ops_opts(a.precision, stream=sptr))
        Vd = torch.empty((a.K, n), dtype=torch.float64, device="cuda")
        mge.mge_embed(ctx.h, h, a.K, a.tol, mge.embed_opts(a.precision, v_on_device=True, stream=sptr), Vd)
        mge.mge_ops_destroy(h)
        mge.mge_graph_destroy(holder.pop("g"))
        C = 16
        idx = torch.from_numpy(np.random.default_rng(6).choice(n, C, replace=False)).cuda()
        C0 = Vd[:, idx].T.contiguous()
        torch.cuda.synchronize()
        steps = {}

        def km():
            steps["s"] = mge.mge_kmeans(ctx.h, Vd, C0, 50, stream=sptr)[2]
        ms = _event_ms(km)
        out["kmeans"] = {"workload": f"the {a.K}-dimensional embedding of that graph (N={n}), {C} clusters from "
                                     "seeded initial rows, Lloyd, at most 50 steps",
                         "ms": ms, "steps": steps["s"], "value": n * steps["s"] / (ms / 1e3),
                         "unit": "point-steps/s"}
        # betweenness centrality and VBC of a 5,000-node manifold graph
        g = mg.manifold_graph(a.shape, 5000, a.knn, a.seed)
        rpd = torch.from_numpy(g.row_ptr).cuda()
        cold = torch.from_numpy(g.col).cuda()
        torch.cuda.synchronize()
        res = {}

        def bc():
            res["v"] = mge.mge_betweenness(ctx.h, g.n, rpd, cold, stream=sptr)[1]
        ms = _event_ms(bc, reps=2)
        out["betweenness"] = {"workload": f"{a.shape} N=5000 {a.knn}-NN graph (nnz {g.nnz}): C_B of every node "
                                          "(all n sources, Brandes) and VBC",
                              "ms": ms, "vbc": res["v"], "value": g.n * g.nnz / (ms / 1e3),
                              "unit": "edge traversals/s (n nnz per call)"}
    return out


# ---------------------------------------------------------------------------------------
# the oracle on the host cores
# ---------------------------------------------------------------------------------------
def oracle_step(a, n, seed):
    """One oracle pass; returns (wall s, process CPU s of all threads, result)."""
    import manifold_graphs as mg
    from oracle import eigen as oe
    from oracle import graph_ops as og
    g = mg.manifold_graph(a.shape, n, a.knn, seed)
    t0, c0 = time.perf_counter(), time.process_time()
    ops = og.from_graph(g, eps_tol=1e-7)
    r = oe.lobpcg(ops.A, ops.b, a.K, tol=a.tol, seed=seed, measure="relative")
    return time.perf_counter() - t0, time.process_time() - c0, r


def cores_used(wall, cpu):
    """Threads the oracle kept busy on average: process CPU time / wall time."""
    return round(cpu / wall, 2) if wall > 0 else None


def oracle_one_thread(a, n):
    """The same oracle step in a child process whose BLAS / OpenMP pools hold one thread."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               BLIS_NUM_THREADS="1")
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-step-only", "--n", str(a.n), "--shape", a.shape,
           "--knn", str(a.knn), "--K", str(a.K), "--tol", repr(a.tol), "--seed", str(a.seed),
           "--cpu-sample-n", str(n)]
    try:
        out = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=600)
        d = json.loads(out.stdout.strip().splitlines()[-1])
        return {"value": n / d["wall_s"], "seconds": d["wall_s"], "cores": cores_used(d["wall_s"], d["cpu_s"])}
    except Exception as e:                      # reported, not fatal: the all-cores figure stands
        return {"error": str(e)[:200]}


def cpu_baseline(a, n, steps=1):
    runs = [oracle_step(a, n, a.seed)[:2] for _ in range(steps)]
    t, c = min(runs)
    return {"value": n / t, "unit": UNIT, "cores": cores_used(t, c), "host_cores": os.cpu_count(),
            "kind": "oracle",
            "sample": f"{a.shape} N={n} {a.knn}-NN K={a.K} tol={a.tol:g}: whole oracle pipeline (FP64 "
                      f"operator build incl. eps by LOBPCG, then FP64 LOBPCG to the same relative residual), "
                      f"{t:.2f} s per graph; cores = process CPU time / wall time",
            "one_thread": oracle_one_thread(a, n)}


def run_reference(a, dist):
    if dist.rank != 0:
        return None
    n = a.cpu_sample_n
    for _ in range(a.warmup):
        oracle_step(a, n, a.seed)
    t0, c0 = time.perf_counter(), time.process_time()
    for _ in range(a.steps):
        oracle_step(a, n, a.seed)
    t, c = time.perf_counter() - t0, time.process_time() - c0
    v = n * a.steps / t
    return {"impl": "reference", "metric": metric(a), "value": v, "unit": UNIT, "n_gpus": dist.world,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * t / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(workload(a), sample=f"N={n} per step (bounded sample of the workload)"),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores_used(t, c), "host_cores": os.cpu_count(),
                             "kind": "oracle",
                             "sample": f"{a.shape} N={n} per step; cores = process CPU time / wall time"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    a = parse()
    if a.oracle_step_only:
        wall, cpu, _ = oracle_step(a, a.cpu_sample_n, a.seed)
        print(json.dumps({"wall_s": wall, "cpu_s": cpu}), flush=True)
        return
    if a.impl == "reference":
        dist = Dist("gloo")
        res = run_reference(a, dist)
        if res is not None:
            print(json.dumps(res), flush=True)
        dist.close()
        return
    dist = Dist("nccl")
    res = run_ours(a, dist)
    if dist.rank == 0:
        # the oracle first, while nothing else of this process keeps the host busy
        if dist.world == 1 and not a.no_cpu_baseline:
            res["cpu_baseline"] = cpu_baseline(a, a.cpu_sample_n)
        if dist.world == 1 and not a.no_batch:
            res["batch"] = run_batch(a)
        if dist.world == 1 and not a.no_serving:
            res["serving"] = run_serving(a)
        if dist.world == 1 and not a.no_sphere_2m:
            res["sphere_2m"] = run_sphere_2m(a)
        if dist.world == 1 and not a.no_extras:
            res.update(run_extras(a))
        print(json.dumps(res), flush=True)
    dist.close()


if __name__ == "__main__":
    main()
