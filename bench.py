#!/usr/bin/env python
"""Benchmark of the PPRviz hot path on GB300.

One step = the whole hot path on the benchmark workload: Chung-Lu graph
n = 10,000, mean degree 20, exponent 2.5, seed 0 (unit weights); graph ingest
and validation (P0), all-pairs FP32 DPPR with the FP64 residual certificate
and refinement to eps = 1e-6 (P1/P2), PDist (P3), then 500 FP32
stress-majorization updates from U[-1,1]^2 with the final stress (P4/P5).

`value` is DPPR entries per second over the whole step (k^2 certified DPPR
entries per step), with inputs already in HBM. `e2e` is the same metric through
the public API with pinned host buffers (CSR, view, PDist round trip, X0 in;
DPPR, PDist, X out), copies inside the timed region.

`--impl reference` times the FP64 CPU oracle on a bounded sample of the same
workload (the reference arm of this benchmark).

`--workload views` measures the batched-views workload instead (not the
default line): 256 SBM views of 50..5,000 nodes, one pprviz_views_batch call
per step (DPPR + PDist + 200 layout updates of every view).

`--workload view2m`: the 8,192-node view of a 2M-node Chung-Lu graph (DPPR /
PDist among the view, then the stress energy and its backward through the
autograd function). `--workload small`: the n = 1,000 FP64 plain-method
workload (DPPR + PDist + 300 FP64 layout updates). `--workload taupush`: Tau-Push
queries (Sec. 4) on the 2M-node Chung-Lu graph, 8 level-1 supernodes of 25
children x 25 leaves per step. `--workload hierarchy`: the Louvain+ hierarchy
(Sec. 5, Appendix A) of the same graph with k = 25. None of these is the
default line.

`--workload dense` measures the dense-view propagation instead (not the
default line): a dense clustered weighted view, n = 20,000, 20 blocks, 15 %
density, lognormal(0, 1) weights, all nodes as the view; one step = all-pairs
DPPR + PDist with the FP64 certificate, every sweep a BF16 x BF16 -> FP32
tensor-core contraction with FP32 refinement (`--dense-precision tf32x3`: the
3xTF32 sweeps; the other mode is timed beside it); the roofline is the tensor
pipe's against the measured BF16 peak (TF32: x the nominal ratio 1.1/2.25).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

ALPHA, EPS = 0.15, 1e-6
WORKLOAD = "chung_lu_n10000_deg20"
L2_FLUSH_BYTES = 512 << 20  # larger than the 126 MB L2


# One launch in PROF_EVERY of the classes launched hundreds of times per step
# is bracketed by CUDA events (every launch of the others): events between all
# launches would serialise them and slow the step being measured.
PROF_EVERY = 16


def max_over_ranks(x, device):
    """The largest x over the ranks of the process group (x itself when there
    is no group or a single rank): the job's time is its slowest rank's."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier_if_group():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def whole_job_rate(units_per_rank_step, steps, world, max_ms):
    """Units per second of the whole job: every rank's units over the slowest
    rank's time (weak scaling: each rank runs its own replica)."""
    return world * steps * units_per_rank_step / (max_ms / 1e3)


def class_share(ktimes, steps):
    """Per class and step: device ms (the timed launches' mean duration x all
    launches) and launches."""
    out = {}
    for c, (ms, cnt, timed) in ktimes.items():
        if cnt and timed:
            out[c] = {"ms": ms / timed * cnt / steps, "launches": cnt / steps, "timed_launches": timed / steps}
    return out


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", "--num-nodes", dest="n", type=int, default=None,
                    help="nodes (default 10000; 20000 with --workload dense); under torchrun use --num-nodes")
    ap.add_argument("--deg", type=float, default=20.0)
    ap.add_argument("--iters", type=int, default=500)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-all-cores", type=int, default=1,
                    help="also time the oracle sample on every host core (1) or not (0)")
    ap.add_argument("--fp64-steps", type=int, default=1,
                    help="timed steps of the plain FP64 GPU path on the same workload (0 = skip)")
    ap.add_argument("--case", action="store_true",
                    help="one untimed pass of the hot path (for profiler command lines)")
    ap.add_argument("--dense-precision", default="bf16", choices=["bf16", "tf32x3"],
                    help="tensor-core sweep operands of --workload dense (the other mode is timed beside it)")
    ap.add_argument("--workload", default="chung_lu", choices=["chung_lu", "dense", "views", "view2m", "small", "taupush", "level", "directed", "metrics", "hierarchy"],
                    help="dense: the dense weighted view on the tensor-core sweeps (--n defaults to 20000); "
                         "views: the 256 batched SBM views; taupush: Tau-Push queries on the 2M-node graph")
    return ap.parse_args()


def run_case(args):
    """One pass of the hot path on the workload, untimed: ingest, FP32 DPPR +
    PDist with certificate, `--iters` layout updates, energy with gradient."""
    import torch
    if args.workload == "dense":
        run_dense_case(args)
        return

    import paper_2112_14944_gb300 as P
    import synth
    n = args.n
    g = synth.chung_lu(n, args.deg, 2.5, seed=0)
    ctx = P.Context(0, torch_stream=True)
    dev = torch.device("cuda", 0)
    rp = torch.from_numpy(g.row_ptr).to(dev)
    col = torch.from_numpy(g.col).to(dev)
    view = torch.arange(n, dtype=torch.int32, device=dev)
    D = torch.empty((n, n), dtype=torch.float32, device=dev)
    Dl = torch.empty_like(D)
    x0 = torch.from_numpy(synth.uniform_x0(n, seed=0)).to(dev)
    xo = torch.empty_like(x0)
    G = ctx.upload(n, rp, col)
    _, _, cert, status = ctx.dppr(G, view, ALPHA, EPS, P.FP32, dppr_out=D, pdist_out=Dl, cert=True)
    st = ctx.stats()
    _, s = ctx.layout(Dl, x0, args.iters, P.FP32, x_out=xo)
    e, _, _ = ctx.energy(Dl, xo, grad_x=True)
    torch.cuda.synchronize()
    print(json.dumps({"case": WORKLOAD, "n": n, "iters": args.iters, "status": status,
                      "max_cert": float(cert.max()), "stress": s, "energy": e, "dppr_stats": st}))


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d["hbm_gbs"], d.get("sm_max_mhz", 2070.0), "measured"
    return 6800.0, 2070.0, "fallback"


def tf32_tflops():
    """Dense TF32 tensor peak: the measured BF16 peak (burst) x the nominal
    TF32/BF16 ratio 1.1/2.25. Returns (TFLOP/s, how it was derived)."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    bf16, kind = 1900.0, "fallback"
    if os.path.exists(p):
        with open(p) as f:
            bf16, kind = json.load(f)["bf16_tflops"], "measured"
    return bf16 * 1.1 / 2.25, f"{kind} bf16_tflops x 1.1/2.25 (nominal TF32/BF16), frac of {kind}"


def config(args, n_gpus):
    return {"workload": WORKLOAD, "graph": "chung-lu", "n": args.n, "mean_degree": args.deg, "exponent": 2.5,
            "seed": 0, "view": "all nodes (k = n)", "alpha": ALPHA, "eps": EPS, "layout_iters": args.iters,
            "propagation": "fp32 chebyshev + fp64 residual certificate + fp32 refinement",
            "layout": "fp32 stress majorization, exact (L^w)^+ solve",
            "l2": "flushed between timed steps (512 MB write)", "parallelism": f"replicas x{n_gpus}"}


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    """Samples nvidia-smi every 200 ms while running."""

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=2)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# --------------------------------------------------------------------------- traffic
def kernel_source_hash(src):
    """sha256 prefix of one kernel's source text: the part of `file` from the
    first occurrence of `begin` up to the next occurrence of `end`."""
    with open(os.path.join(ROOT, "paper_2112_14944_gb300", "csrc", src["file"])) as fh:
        text = fh.read()
    a = text.find(src["begin"])
    if a < 0:
        return None
    b = text.find(src["end"], a + len(src["begin"]))
    body = text[a:b if b > a else len(text)]
    return hashlib.sha256(body.encode()).hexdigest()[:16]


def measured_traffic(cls):
    """DRAM bytes per launch of a kernel class from the committed ncu summary
    (profiles/traffic.json), or None when absent or when the kernel's source
    text has changed since the counters were taken."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f).get(cls)
    if not d:
        return None
    if d.get("source_hash") != kernel_source_hash(d["src"]):
        return None
    return d.get("dram_bytes_per_launch")


# --------------------------------------------------------------------------- reference arm
def cpu_oracle_rows(g, src, n_clamp=None):
    """FP64 oracle on a bounded sample: the DPPR rows pi_d(s, .) of the
    sources `src` and the PDist rows they fix (power iteration to
    (1 - alpha)^(t+1) <= 1e-15 for rows and columns). Returns (DPPR rows,
    PDist rows, z rows, seconds)."""
    import oracle as O
    t0 = time.perf_counter()
    Pm = O.transition_matrix(g.n, g.row_ptr, g.col, g.weight)
    d = O.degrees(g.n, g.row_ptr, g.col, g.weight)
    rows = O.ppr_rows(Pm, src, ALPHA)
    cols = O.ppr_cols(Pm, src, ALPHA)
    D = O.dppr_rows(rows, d, src)
    Dc = (d[:, None] * cols).T
    z = D + Dc
    Dl = O.pdist_from_z(z, g.n if n_clamp is None else n_clamp)
    Dl[np.arange(len(src)), src] = 0.0
    return D, Dl, z, time.perf_counter() - t0


def cpu_oracle_sample(g, n_src, seed=1):
    """The oracle's DPPR rows of n_src seeded sources and the PDist rows they
    fix, on one thread. Returns (entries, seconds)."""
    import synth
    src = synth.sample_view(g.n, n_src, seed=seed)
    _, _, _, t = cpu_oracle_rows(g, src)
    return n_src * g.n, t


def _oracle_worker(args):
    n, row_ptr, col, weight, src = args
    import synth
    g = synth.Graph(n, row_ptr, col, weight)
    _, _, _, t = cpu_oracle_rows(g, src)
    return len(src) * n, t


def cpu_oracle_all_cores(g, n_src_per_core, seed=7):
    """The same oracle sample on every host core: one process per core
    (spawned, so it is safe after CUDA is initialised), each computing the
    rows of its own n_src_per_core seeded sources. Returns (entries, wall
    seconds of the parallel part, cores)."""
    import multiprocessing as mp

    import synth
    cores = os.cpu_count() or 1
    src = synth.sample_view(g.n, min(g.n, cores * n_src_per_core), seed=seed)
    chunks = [src[i::cores] for i in range(cores)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores, initializer=_pool_init) as pool:
        pool.map(_pool_ping, range(cores))  # workers started and imported before the clock
        t0 = time.perf_counter()
        res = pool.map(_oracle_worker, [(g.n, g.row_ptr, g.col, g.weight, c) for c in chunks if len(c)])
        wall = time.perf_counter() - t0
    return sum(e for e, _ in res), wall, cores


def _pool_init():
    # one BLAS thread per worker: the pool itself is the parallelism
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    sys.path.insert(0, ROOT)
    import oracle  # noqa: F401
    import synth  # noqa: F401


def _pool_ping(i):
    return i


def oracle_errors(g, src, D, Dl, cert):
    """Per-result error of the GPU outputs against the oracle's rows of the
    sampled sources (the CPU-baseline sample): DPPR max-abs and
    max-abs / max(1, |ref|), PDist max-abs and the largest excess over the
    certified PDist tolerance (<= 0 when every entry passes)."""
    import math
    Dref, Dlref, z, _ = cpu_oracle_rows(g, src)
    Dg = np.asarray(D, dtype=np.float64)
    Dlg = np.asarray(Dl, dtype=np.float64)
    e_d = np.abs(Dg - Dref)
    e_l = np.abs(Dlg - Dlref)
    # the certified PDist tolerance of Eq. (1): 1e-5 + (c_s + c_t) / max(z - c_s - c_t, e / n^2)
    # with z = pi_d(s, t) + pi_d(t, s) from the oracle's rows and columns
    c = np.asarray(cert, dtype=np.float64)
    cc = c[src][:, None] + c[None, :]
    tol = 1e-5 + cc / np.maximum(z - cc, math.e / float(g.n) ** 2)
    tol[np.arange(len(src)), src] = 1e-5
    return {"sample_sources": len(src), "dppr_max_abs": float(e_d.max()),
            "dppr_max_abs_over_max1": float((e_d / np.maximum(1.0, np.abs(Dref))).max()),
            "pdist_max_abs": float(e_l.max()), "pdist_certified_gate_excess": float((e_l - tol).max()),
            "max_cert": float(c.max())}


def layout_update_error_bound(Dl, X0, X1):
    """A bound on the error of one GPU stress-majorization update that needs
    no oracle: with b = L^Y(X0) X0 and r = L^w X1 - b (both in FP64 on the
    host, from the GPU's PDist), the exact centred update X* satisfies
    |X1 - X*|_F <= |r|_F / lambda_2(L^w), and lambda_2(L^w) >= k w_min for
    the complete-graph Laplacian L^w with weights w_ij = 1 / Delta_ij^2 >= w_min
    (Appendix A.1, Eq. (10)). Returns (that bound, and the first Jacobi
    estimate max_i |r_i| / L^w_ii of the error), both over max(1, max|X1|)."""
    D = np.asarray(Dl, dtype=np.float64)
    k = D.shape[0]
    X0 = np.asarray(X0, dtype=np.float64)
    X1 = np.asarray(X1, dtype=np.float64)
    r = np.zeros((k, 2))
    diag = np.zeros(k)
    wmin = np.inf
    for a in range(0, k, 1024):
        Db = D[a:a + 1024]
        off = np.ones_like(Db, dtype=bool)
        off[np.arange(len(Db)), np.arange(a, a + len(Db))] = False
        W = np.where(off, 1.0 / np.where(off, Db, 1.0) ** 2, 0.0)
        wmin = min(wmin, float(W[off].min()))
        diff0 = X0[a:a + len(Db), None, :] - X0[None, :, :]
        d0 = np.sqrt((diff0 ** 2).sum(-1))
        LY = np.where(off & (d0 > 0), 1.0 / (np.where(off, Db, 1.0) * np.where(d0 > 0, d0, 1.0)), 0.0)
        b = (LY[:, :, None] * diff0).sum(1)
        lw = (W[:, :, None] * (X1[a:a + len(Db), None, :] - X1[None, :, :])).sum(1)
        r[a:a + len(Db)] = lw - b
        diag[a:a + len(Db)] = W.sum(1)
    scale = max(1.0, float(np.abs(X1).max()))
    bound = float(np.sqrt((r ** 2).sum()) / (k * wmin))
    jac = float((np.abs(r) / diag[:, None]).max())
    return bound / scale, jac / scale


def run_reference(args, rank, world):
    if rank != 0:
        return
    import synth
    g = synth.chung_lu(args.n, args.deg, 2.5, seed=0)
    n_src = 16
    for _ in range(args.warmup):
        cpu_oracle_sample(g, 4)
    times, ents = [], 0
    for s in range(args.steps):
        e, t = cpu_oracle_sample(g, n_src, seed=100 + s)
        times.append(t)
        ents += e
    total = sum(times)
    value = ents / total
    line = {
        "impl": "reference", "metric": "DPPR entries/s at n=10k, err<=1e-6 vs FP64; layout iters/s; % HBM roofline",
        "value": value, "unit": "entries/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config(args, world),
        "cpu_baseline": {"value": value, "unit": "entries/s", "cores": 1, "kind": "oracle",
                         "sample": f"{n_src} seeded sources per step: DPPR rows and PDist rows by FP64 power "
                                   f"iteration to (1-alpha)^(t+1) <= 1e-15"},
        "e2e": {"value": value, "unit": "entries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- dense views
DENSE_WORKLOAD = "dense_clustered_weighted_n20000_d15"


def dense_graph(n):
    import synth
    return synth.dense_clustered(n, blocks=20, density=0.15, seed=0)


def run_dense_case(args):
    """One untimed all-pairs DPPR + PDist on the dense weighted view."""
    import torch

    import paper_2112_14944_gb300 as P
    n = args.n
    g = dense_graph(n)
    ctx = P.Context(0, torch_stream=True)
    dev = torch.device("cuda", 0)
    G = ctx.upload(n, torch.from_numpy(g.row_ptr).to(dev), torch.from_numpy(g.col).to(dev),
                   torch.from_numpy(g.weight).to(dev))
    view = torch.arange(n, dtype=torch.int32, device=dev)
    D = torch.empty((n, n), dtype=torch.float32, device=dev)
    Dl = torch.empty_like(D)
    _, _, cert, status = ctx.dppr(G, view, ALPHA, EPS, P.FP32, dppr_out=D, pdist_out=Dl, cert=True)
    torch.cuda.synchronize()
    print(json.dumps({"case": DENSE_WORKLOAD, "n": n, "nnz": int(g.nnz), "status": status,
                      "max_cert": float(cert.max()), "dppr_stats": ctx.stats()}))


def run_dense(args, rank, world, local_rank):
    """The dense weighted view: all-pairs DPPR + PDist with the FP64
    certificate, every sweep a tensor-core contraction. The line's mode is
    BF16 x BF16 -> FP32 (kind::f16) with FP32 refinement; the 3xTF32 mode is
    timed beside it on the same view."""
    import torch

    import paper_2112_14944_gb300 as P
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    n = args.n
    g = dense_graph(n)
    ctx = P.Context(local_rank, torch_stream=True)
    stream = ctx._stream
    rp = torch.from_numpy(g.row_ptr).to(dev)
    col = torch.from_numpy(g.col).to(dev)
    w = torch.from_numpy(g.weight).to(dev)
    view = torch.arange(n, dtype=torch.int32, device=dev)
    D = torch.empty((n, n), dtype=torch.float32, device=dev)
    Dl = torch.empty_like(D)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    G = ctx.upload(n, rp, col, w)
    modes = {"bf16": P.FP32_BF16TC, "tf32x3": P.FP32_TC}
    main = args.dense_precision
    other = "tf32x3" if main == "bf16" else "bf16"

    def step(prec):
        _, _, cert, status = ctx.dppr(G, view, ALPHA, EPS, prec, dppr_out=D, pdist_out=Dl, cert=True)
        return ctx.stats(), status, float(cert.max())

    def timed(prec, steps, prof):
        if prof:
            ctx.profile(PROF_EVERY)
        ms, flops, launches, sweeps, stats, sts, certs = [], 0.0, 0, 0, None, [], []
        for _ in range(steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            stats, st, cm = step(prec)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            sts.append(st)
            certs.append(cm)
            flops += stats["flops_dense"]
            launches += stats["kernel_launches"]
            sweeps += stats["sweeps_main"] + stats["sweeps_refine"]
        kt = ctx.kernel_times() if prof else None
        if prof:
            ctx.profile(False)
        assert all(x == 0 for x in sts) and max(certs) <= EPS, (sts, max(certs))
        return ms, flops, launches, sweeps, stats, kt, max(certs)

    for _ in range(args.warmup):
        step(modes[main])
    step(modes[other])
    torch.cuda.synchronize()
    barrier_if_group()
    torch.cuda.synchronize()
    sampler = ClockSampler(local_rank)
    sampler.start()
    ms, flops, launches, sweeps, stats, ktimes, cmax = timed(modes[main], args.steps, True)
    torch.cuda.synchronize()
    sampler.stop()
    total = max_over_ranks(sum(ms), dev)
    ms_o, fl_o, _, sw_o, st_o, _, cm_o = timed(modes[other], 1, False)
    if rank != 0:
        return
    entries = float(n) * n
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    bf16, kind = 1900.0, "fallback"
    if os.path.exists(pk):
        with open(pk) as f:
            bf16, kind = json.load(f)["bf16_tflops"], "measured"
    tf32 = bf16 * 1.1 / 2.25
    peak = bf16 if main == "bf16" else tf32
    sw_ms, sw_all, sw_n = ktimes["sweep"]
    ach = flops / sw_all * sw_n / (sw_ms / 1e3) / 1e12  # flops of the timed launches / their time
    issued = 1 if main == "bf16" else 3
    roof = {"kernel": ("tensor-core sweep (k_dsweep_tc, BF16 x BF16 -> FP32 tcgen05.mma kind::f16)" if main == "bf16"
                       else "tensor-core sweep (k_dsweep_tc, 3xTF32 tcgen05.mma kind::tf32)"),
            "bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
            "executed_tflops": issued * ach, "executed_frac": issued * ach / peak,
            "launches": sw_all, "timed_launches": sw_n, "avg_launch_us": 1e3 * sw_ms / max(1, sw_n),
            "alg_flops_per_launch": flops / max(1, sw_all), "traffic": measured_traffic("dsweep"),
            "peak_kind": (f"{kind} bf16_tflops, frac of {kind}" if main == "bf16" else
                          f"{kind} bf16_tflops x 1.1/2.25 (nominal TF32/BF16), frac of {kind}")}
    share = class_share(ktimes, args.steps)
    line = {
        "metric": "DPPR entries/s, dense weighted view n=20k, err<=1e-6 vs FP64 (tensor-core sweeps)",
        "value": whole_job_rate(entries, args.steps, world, total), "unit": "entries/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16/f32/f64" if main == "bf16" else "tf32x3/f32/f64",
        "data": "synthetic",
        "config": {"workload": DENSE_WORKLOAD, "graph": "dense clustered SBM, lognormal(0,1) weights", "n": n,
                   "nnz": int(g.nnz), "blocks": 20, "density": 0.15, "seed": 0, "view": "all nodes (k = n)",
                   "alpha": ALPHA, "eps": EPS,
                   "propagation": (f"fp32 chebyshev on {main} tensor-core sweeps + fp64 residual certificate "
                                   "+ fp32 refinement"),
                   "l2": "flushed between timed steps (512 MB write)", "parallelism": f"replicas x{world}"},
        "sweeps_per_step": sweeps / args.steps,
        "refine_passes_per_step": stats["refine_passes"] if stats else None,
        "residual_passes_per_step": stats["residual_passes"] if stats else None,
        "max_cert": cmax, "roofline": roof, "kernel_share": share, "gpu_launches": int(launches),
        "other_mode": {"mode": other, "ms_per_step": statistics.mean(ms_o), "sweeps_per_step": sw_o,
                       "refine_passes": st_o["refine_passes"], "residual_passes": st_o["residual_passes"],
                       "max_cert": cm_o},
        "clocks": sampler.summary(),
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- batched views
VIEWS_WORKLOAD = "sbm_views_256_n50_5000"


def run_views(args, rank, world, local_rank):
    """The batched-views workload: 256 SBM views (n_v ~ U{50..5000}, 4..16
    blocks, p_in 0.1, p_out 0.002, seed 0); one step = one pprviz_views_batch
    call on device buffers: all-pairs DPPR + PDist of every view (certified to
    eps) and 200 FP32 layout updates of every view."""
    import torch

    import paper_2112_14944_gb300 as P
    import synth
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    graphs = synth.sbm_views(256, seed=0)
    ctx = P.Context(local_rank, torch_stream=True)
    stream = ctx._stream
    G = [ctx.upload_graph(g) for g in graphs]
    x0 = torch.from_numpy(np.concatenate([synth.uniform_x0(g.n, seed=1000 + i)
                                          for i, g in enumerate(graphs)])).to(dev)
    entries = float(sum(g.n * g.n for g in graphs))
    iters = 200
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def step():
        _, _, _, _, cert = ctx.views_batch(G, x0, ALPHA, EPS, iters, want_pdist=True, want_cert=True)
        assert np.all(cert <= EPS), cert.max()
        return ctx.stats()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier_if_group()
    torch.cuda.synchronize()
    # timed steps run as the user runs them (layout updates as one CUDA graph,
    # kernel timing off); the kernel shares come from one more step, after
    # the timed region, with kernel timing on (updates launched one by one)
    sampler = ClockSampler(local_rank)
    sampler.start()
    ms, launches, stats = [], 0, None
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        stats = step()
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
        launches += stats["kernel_launches"]
    torch.cuda.synchronize()
    sampler.stop()
    graphed = bool(stats and stats.get("graph_launched"))
    ctx.profile(PROF_EVERY)
    with torch.cuda.stream(stream):
        flush.zero_()
    step()
    ktimes = ctx.kernel_times()
    ctx.profile(False)
    total = sum(ms)
    total = max_over_ranks(total, dev)
    if rank != 0:
        return
    line = {
        "metric": "DPPR entries/s, 256 batched SBM views (DPPR + PDist + 200 layout updates each)",
        "value": whole_job_rate(entries, args.steps, world, total), "unit": "entries/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": VIEWS_WORKLOAD, "views": 256, "n_range": [50, 5000], "blocks": [4, 16],
                   "p_in": 0.1, "p_out": 0.002, "seed": 0, "sum_n": int(sum(g.n for g in graphs)),
                   "sum_n2": int(entries), "alpha": ALPHA, "eps": EPS, "layout_iters": iters,
                   "l2": "flushed between timed steps (512 MB write)", "parallelism": f"replicas x{world}"},
        "views_stats": {k: stats[k] for k in ("groups", "sweeps_main", "sweeps_refine", "residual_passes",
                                              "max_cert", "source_group")} if stats else None,
        "layout_updates_as_cuda_graph": graphed,
        "kernel_share": class_share(ktimes, 1),
        "kernel_share_from": "one extra step after the timed region, kernel timing on, updates launched one by one",
        "gpu_launches": int(launches),
        "clocks": sampler.summary(),
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- Tau-Push queries
TAUPUSH_WORKLOAD = "chung_lu_n2000000_deg10_taupush_level1_k25x25"
TP_QUERIES = 8


def run_taupush(args, rank, world, local_rank):
    """Tau-Push queries (Sec. 4, Algorithm 1) on the Chung-Lu graph of
    n = 2,000,000 nodes (mean degree 10, exponent 2.5, seed 0). A query is a
    level-1 supernode of k = 25 children of 25 leaves each, drawn uniformly
    (the randomly chosen supernode of the paper's expected-cost analysis),
    with the paper's eps = 1 - 1/e, delta = 1 / (10 k) and tau = 1 / sqrt(k n).
    One step = 8 queries (seeds 1000..1007); leaf sets, the DPR index and the
    outputs are resident on the device. The DPR index is built once, before
    the timed region, and timed on its own."""
    import math

    import torch

    import oracle as O
    import paper_2112_14944_gb300 as P
    import synth
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    g = synth.chung_lu(2_000_000, 10, 2.5, seed=0)
    k, per = 25, 25
    eps_p, delta = 1 - 1 / math.e, 1.0 / (10 * k)
    ctx = P.Context(local_rank, torch_stream=True)
    stream = ctx._stream
    G = ctx.upload_graph(g)
    dpr = torch.empty(g.n, dtype=torch.float64, device=dev)
    ctx.dpr(G, ALPHA, 1e-12, out=dpr)  # warm-up of the index build
    torch.cuda.synchronize()
    i0, i1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    i0.record(stream)
    _, dpr_cert = ctx.dpr(G, ALPHA, 1e-12, out=dpr)
    i1.record(stream)
    i1.synchronize()
    index_ms = i0.elapsed_time(i1)
    qs = [synth.random_leaf_sets(g.n, [per] * k, seed=1000 + q) for q in range(TP_QUERIES)]
    qd = [(torch.from_numpy(a).to(dev), torch.from_numpy(b).to(dev)) for a, b in qs]
    outs = [(torch.empty((k, k), dtype=torch.float64, device=dev),
             torch.empty((k, k), dtype=torch.float64, device=dev)) for _ in qs]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def step():
        infos, launches = [], 0
        for (pd, idd), (o, po) in zip(qd, outs):
            _, _, info = ctx.tau_push(G, pd, idd, dpr, ALPHA, eps_p, delta, 0.0, ldppr_out=o, pdist_out=po)
            infos.append(info)
            launches += ctx.stats()["kernel_launches"]
        return infos, launches

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier_if_group()
    torch.cuda.synchronize()
    sampler = ClockSampler(local_rank)
    sampler.start()
    ms, launches, infos = [], 0, None
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        infos, nl = step()
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
        launches += nl
    torch.cuda.synchronize()
    sampler.stop()
    total = max_over_ranks(sum(ms), dev)
    # kernel shares: one more step with kernel timing on (every launch timed)
    ctx.profile(1)
    with torch.cuda.stream(stream):
        flush.zero_()
    step()
    ktimes = ctx.kernel_times()
    ctx.profile(False)
    # end to end through the public API with host buffers: each query copies
    # its leaf arrays and the DPR index in and its DPPR and PDist out
    dpr_h = dpr.cpu().numpy()
    e2e_ms = []
    for _ in range(max(1, min(args.steps, 3))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for a, b in qs:
            ctx.tau_push(G, a, b, dpr_h, ALPHA, eps_p, delta, 0.0)
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
    h2d = sum(a.nbytes + b.nbytes for a, b in qs) + TP_QUERIES * dpr_h.nbytes
    d2h = TP_QUERIES * 2 * k * k * 8
    if rank != 0:
        return
    hbm, _, peak_kind = peaks()
    units = sum(i["fwd_edges"] + i["bwd_edges"] for i in infos)
    takes = sum(i["fwd_pushes"] + i["bwd_pushes"] for i in infos)
    push_ms, push_n, _ = ktimes["push"]
    # algorithmic bytes: per unit (an edge times a taken residue) the column
    # index (4 B) and the residue's read-modify-write (8 + 8 B); per taken
    # residue its read and zeroing (8 + 8 B) and its (slot, share) pair (16 B)
    alg = 20.0 * units + 32.0 * takes
    ach = alg / (push_ms / 1e3) / 1e9 if push_ms else None
    roof = {"kernel": "Tau-Push rounds (k_tp_push + k_tp_collect_front), FP64 atomic reductions at random nodes",
            "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm if ach else None,
            "launches": push_n, "alg_bytes_per_step": alg, "alg_bytes_note": "20 B per unit + 32 B per taken residue",
            "device_ms_per_step": push_ms, "traffic": None,
            "peak_kind": f"{peak_kind} hbm_gbs (copy bandwidth), frac of {peak_kind}"}
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        # the oracle's GFP (Algorithm 2, sequential pushes) from the first child
        # of the first query, scaled to a whole query (k children)
        Pm = O.transition_matrix(g.n, g.row_ptr, g.col)
        d = O.degrees(g.n, g.row_ptr, g.col)
        a, b = qs[0]
        leaf_sets = [b[a[i]:a[i + 1]].astype(np.int64) for i in range(k)]
        r_max = eps_p * delta / (d.sum() * (1 / math.sqrt(k * g.n)))
        t0 = time.perf_counter()
        O.gfp(Pm, d, leaf_sets, 0, ALPHA, r_max)
        t_src = time.perf_counter() - t0
        cpu = {"value": 1.0 / (t_src * k), "unit": "queries/s", "cores": 1, "kind": "oracle",
               "sample": f"GFP (sequential pushes, pure Python) from 1 of the 25 children of query 0 "
                         f"({t_src:.1f} s), times 25 for a query; the backward phase refines no target here"}
    # error of query 0's first row against the oracle's group-start power
    # iteration (exact to 1e-9 of the walk mass), with Lemma 2's bound
    a, b = qs[0]
    leaf_sets = [b[a[i]:a[i + 1]].astype(np.int64) for i in range(k)]
    Pm = O.transition_matrix(g.n, g.row_ptr, g.col)
    d = O.degrees(g.n, g.row_ptr, g.col)
    exact = O.level_dppr_rows_power(Pm, d, leaf_sets, [0], ALPHA, tol=1e-9)[0]
    est = outs[0][0][0].cpu().numpy()
    tau_j = np.array([d[F].mean() for F in leaf_sets]) / d.sum()
    bound = infos[0]["r_max"] * d.sum() * tau_j
    err = exact - est
    errors = {"row": 0, "max_underestimate": float(err.max()), "min_underestimate": float(err.min()),
              "lemma2_bound_max": float(bound.max()), "within_bound": bool(np.all(err <= bound + 1e-9)),
              "oracle_tol": 1e-9}
    q_per_step = float(TP_QUERIES)
    e2e_rate = TP_QUERIES / (statistics.mean(e2e_ms) / 1e3)
    line = {
        "metric": "Tau-Push queries/s, level-1 supernode (25 children x 25 leaves), 2M-node power-law graph",
        "value": whole_job_rate(q_per_step, args.steps, world, total), "unit": "queries/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps,
        "ms_per_query": total / args.steps / TP_QUERIES, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": TAUPUSH_WORKLOAD, "graph": "chung-lu", "n": g.n, "nnz": int(g.nnz),
                   "mean_degree": 10, "exponent": 2.5, "seed": 0, "queries_per_step": TP_QUERIES,
                   "query": "k = 25 children x 25 leaves, uniform without replacement (seeds 1000..1007)",
                   "alpha": ALPHA, "eps": eps_p, "delta": delta, "tau": 1 / math.sqrt(k * g.n),
                   "l2": "flushed between timed steps (512 MB write)", "parallelism": f"replicas x{world}"},
        "index": {"dpr_ms": index_ms, "dpr_l1_bound": dpr_cert},
        "per_query": {"rounds": statistics.mean(i["fwd_rounds"] + i["bwd_rounds"] for i in infos),
                      "taken_residues": takes / TP_QUERIES, "units": units / TP_QUERIES,
                      "backward_targets": statistics.mean(i["backward_targets"] for i in infos)},
        "roofline": roof, "errors": errors,
        "kernel_share": class_share(ktimes, 1),
        "kernel_share_from": "one extra step after the timed region, every launch timed",
        "gpu_launches": int(launches),
        "e2e": {"value": e2e_rate, "unit": "queries/s", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": d2h},
        "cpu_baseline": cpu, "clocks": sampler.summary(),
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- level-l DPPR, directed, metrics
LEVEL_WORKLOAD = "chung_lu_n2000000_deg10_level1_k25x25"
DIRECTED_WORKLOAD = "directed_chung_lu_n10000_deg20"
METRICS_WORKLOAD = "layout_n10000_nd_ulcv"


def _timed_steps(args, stream, flush, step):
    """Warm-up, then args.steps steps between CUDA events on `stream` with the
    L2 flushed before each and the clocks sampled; returns (ms per step list,
    last step's result, clock summary)."""
    import torch
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier_if_group()
    torch.cuda.synchronize()
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    ms, out = [], None
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = step()
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    sampler.stop()
    return ms, out, sampler.summary()


def run_level(args, rank, world, local_rank):
    """Exact level-l DPPR (Sec. 3.2, Definition 2, Eq. (2)) for the Tau-Push
    queries of `--workload taupush`: the 2M-node Chung-Lu graph, 8 level-1
    supernodes of 25 children x 25 leaves (seeds 1000..1007); one certified
    FP32 propagation per child from its group start, eps = 1e-6; one step =
    the 8 queries."""
    import torch

    import oracle as O
    import paper_2112_14944_gb300 as P
    import synth
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    g = synth.chung_lu(2_000_000, 10, 2.5, seed=0)
    k = 25
    ctx = P.Context(local_rank, torch_stream=True)
    stream = ctx._stream
    G = ctx.upload_graph(g)
    qs = [synth.random_leaf_sets(g.n, [25] * k, seed=1000 + q) for q in range(TP_QUERIES)]
    sets = [[b[a[i]:a[i + 1]] for i in range(k)] for a, b in qs]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    state = {}

    def step():
        outs, launches, sweeps, bsweep, cmax = [], 0, 0, 0.0, 0.0
        for ls in sets:
            D, _, cert, st = ctx.level_dppr(G, ls, ALPHA, EPS, out64=True)
            assert st == 0 and cert.max() <= EPS
            s = ctx.stats()
            launches += s["kernel_launches"]
            sweeps += s["sweeps_main"] + s["sweeps_refine"]
            cmax = max(cmax, float(cert.max()))
            outs.append(D)
        # 12 B per (node, source) and sweep: y_k and y_k-1 read, y_k+1 written
        state.update(launches=launches, sweeps=sweeps, bytes_per_sweep=12.0 * g.n * s["source_group"], cmax=cmax)
        return outs

    ctx.profile(PROF_EVERY)
    ms, outs, clocks = _timed_steps(args, stream, flush, step)
    ktimes = ctx.kernel_times()
    ctx.profile(False)
    total = max_over_ranks(sum(ms), dev)
    if rank != 0:
        return
    hbm, _, peak_kind = peaks()
    sw_ms, sw_all, sw_n = ktimes["sweep"]
    per = state["bytes_per_sweep"]
    ach = per / (sw_ms / max(1, sw_n) / 1e3) / 1e9 if sw_n else None
    roof = {"kernel": "propagation sweep (k_sweep_sp): the [2M][128] state streams from HBM", "bound": "hbm",
            "alg_bytes_per_launch": per,
            "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm if ach else None,
            "avg_launch_us": 1e3 * sw_ms / max(1, sw_n), "traffic": None,
            "peak_kind": f"{peak_kind} hbm_gbs (copy bandwidth), frac of {peak_kind}"}
    # query 0, row 0 against the oracle's group-start power iteration
    Pm = O.transition_matrix(g.n, g.row_ptr, g.col)
    d = O.degrees(g.n, g.row_ptr, g.col)
    exact = O.level_dppr_rows_power(Pm, d, [x.astype(np.int64) for x in sets[0]], [0], ALPHA, tol=1e-12)[0]
    err = float(np.abs(outs[0][0] - exact).max())
    line = {
        "metric": "exact level-l DPPR queries/s (25 children x 25 leaves, eps 1e-6), 2M-node power-law graph",
        "value": whole_job_rate(float(TP_QUERIES), args.steps, world, total), "unit": "queries/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps,
        "ms_per_query": total / args.steps / TP_QUERIES, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": LEVEL_WORKLOAD, "graph": "chung-lu", "n": g.n, "mean_degree": 10, "exponent": 2.5,
                   "seed": 0, "queries_per_step": TP_QUERIES, "query": "the taupush workload's queries",
                   "alpha": ALPHA, "eps": EPS, "l2": "flushed between timed steps (512 MB write)",
                   "parallelism": f"replicas x{world}"},
        "sweeps_per_step": state["sweeps"] / 1.0, "max_cert": state["cmax"],
        "errors": {"query0_row0_max_abs_vs_oracle": err, "oracle_tol": 1e-12},
        "roofline": roof, "kernel_share": class_share(ktimes, args.steps + args.warmup),
        "gpu_launches": int(state["launches"] * args.steps), "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


def run_directed(args, rank, world, local_rank):
    """Directed input (Sec. 2.1): the n = 10k Chung-Lu graph (mean degree 20,
    seed 0) made directed (each edge kept both ways with probability 0.3,
    otherwise one random way; 2 % of the nodes dangling; seed 0); all-pairs
    FP32 DPPR + PDist with the FP64 certificate (power sweeps: the walk is not
    reversible), eps = 1e-6."""
    import torch

    import paper_2112_14944_gb300 as P
    import synth
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    g = synth.directed_from(synth.chung_lu(10000, 20, 2.5, seed=0), p_both=0.3, dangling=0.02, seed=0)
    n = g.n
    ctx = P.Context(local_rank, torch_stream=True)
    stream = ctx._stream
    G = ctx.upload_graph(g)
    view = torch.arange(n, dtype=torch.int32, device=dev)
    D = torch.empty((n, n), dtype=torch.float32, device=dev)
    Dl = torch.empty_like(D)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    state = {}

    def step():
        _, _, cert, st = ctx.dppr(G, view, ALPHA, EPS, P.FP32, dppr_out=D, pdist_out=Dl, cert=True)
        s = ctx.stats()
        state.update(st=st, cert=cert, launches=s["kernel_launches"], sweeps=s["sweeps_main"] + s["sweeps_refine"],
                     bsweep=s["bytes_sweep"])
        return st

    ctx.profile(PROF_EVERY)
    ms, _, clocks = _timed_steps(args, stream, flush, step)
    ktimes = ctx.kernel_times()
    ctx.profile(False)
    assert state["st"] == 0 and float(state["cert"].max()) <= EPS
    total = max_over_ranks(sum(ms), dev)
    errors = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        src = synth.sample_view(n, 16, seed=1)
        errors = oracle_errors(g, src, D[torch.from_numpy(src).to(dev).long()].cpu().numpy(),
                               Dl[torch.from_numpy(src).to(dev).long()].cpu().numpy(), state["cert"])
    if rank != 0:
        return
    hbm, _, peak_kind = peaks()
    sw_ms, sw_all, sw_n = ktimes["sweep"]
    per = state["bsweep"] / max(1, sw_all / (args.steps + args.warmup))
    ach = per / (sw_ms / max(1, sw_n) / 1e3) / 1e9 if sw_n else None
    roof = {"kernel": "propagation sweep (k_sweep_sp, power sweeps over the pull CSR)", "bound": "hbm",
            "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm if ach else None,
            "avg_launch_us": 1e3 * sw_ms / max(1, sw_n), "traffic": None,
            "peak_kind": f"{peak_kind} hbm_gbs (copy bandwidth), frac of {peak_kind}"}
    line = {
        "metric": "DPPR entries/s, directed Chung-Lu n=10k, err<=1e-6 vs FP64 (DPPR + PDist)",
        "value": whole_job_rate(float(n) * n, args.steps, world, total), "unit": "entries/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": DIRECTED_WORKLOAD, "graph": "directed chung-lu", "n": n, "nnz": int(g.nnz),
                   "p_both": 0.3, "dangling": 0.02, "seed": 0, "alpha": ALPHA, "eps": EPS,
                   "view": "all nodes (k = n)", "l2": "flushed between timed steps (512 MB write)",
                   "parallelism": f"replicas x{world}"},
        "sweeps_per_step": state["sweeps"], "max_cert": float(state["cert"].max()), "errors": errors,
        "roofline": roof, "kernel_share": class_share(ktimes, args.steps + args.warmup),
        "gpu_launches": int(state["launches"] * args.steps), "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


def run_metrics(args, rank, world, local_rank):
    """ND and ULCV (Sec. 2) of a 10,000-node layout: U[-1,1]^2 coordinates
    (seed 0) of the n = 10k Chung-Lu graph (mean degree 20, seed 0); ND over
    the 5.0e7 pairs, ULCV over the 99,665 edges, FP64 arithmetic; one step =
    one pprviz_layout_metrics call on device buffers."""
    import torch

    import oracle as O
    import paper_2112_14944_gb300 as P
    import synth
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    g = synth.chung_lu(10000, 20, 2.5, seed=0)
    n = g.n
    ctx = P.Context(local_rank, torch_stream=True)
    stream = ctx._stream
    G = ctx.upload_graph(g)
    xh = synth.uniform_x0(n, seed=0)
    x = torch.from_numpy(xh).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    ms, res, clocks = _timed_steps(args, stream, flush, lambda: ctx.layout_metrics(x, G))
    launches = ctx.stats()["kernel_launches"]
    total = max_over_ranks(sum(ms), dev)
    if rank != 0:
        return
    nd, ul = res
    iu = np.triu_indices(n, 1)
    e = np.stack([np.repeat(np.arange(n), np.diff(g.row_ptr)), g.col], 1)
    e = e[e[:, 0] < e[:, 1]]
    nd_ref = O.node_distribution(xh.astype(np.float64))
    ul_ref = O.ulcv(xh.astype(np.float64), e)
    pairs = n * (n - 1) / 2
    fp64 = 1250.0  # GB300 nominal FP64 (vector) TFLOP/s x 1000 = GFLOP/s
    ach = 7.0 * pairs / (total / args.steps / 1e3) / 1e9
    line = {
        "metric": "layout metrics (ND over all pairs + ULCV over the edges) of a 10,000-node layout, ms per call",
        "value": total / args.steps, "unit": "ms", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total / args.steps, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": METRICS_WORKLOAD, "graph": "chung-lu", "n": n, "pairs": int(pairs), "edges": int(len(e)),
                   "coordinates": "U[-1,1]^2 (seed 0)", "l2": "flushed between timed steps (512 MB write)",
                   "parallelism": f"replicas x{world}"},
        "errors": {"nd_rel": abs(nd - nd_ref) / abs(nd_ref), "ulcv_rel": abs(ul - ul_ref) / abs(ul_ref)},
        "roofline": {"kernel": "k_nd (FP64 per pair: 2 sub, 2 mul, add, divide, accumulate)", "bound": "alu",
                     "achieved": ach, "peak": fp64, "unit": "GFLOP/s (FP64, 7 per pair)", "frac": ach / fp64,
                     "peak_kind": "nominal FP64 rate of the part (1.25 TFLOP/s), not measured", "traffic": None},
        "gpu_launches": int(launches * args.steps), "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- Louvain+ hierarchy
HIER_WORKLOAD = "chung_lu_n2000000_deg10_louvain_plus_k25"


def run_hierarchy(args, rank, world, local_rank):
    """The Louvain+ supergraph hierarchy (Sec. 5 preprocessing; Appendix A)
    of the 2M-node Chung-Lu graph of the Tau-Push workload (mean degree 10,
    exponent 2.5, seed 0), k = 25; one step = one pprviz_louvain_plus call on
    the resident graph, its parent arrays read back to the host (part of the
    call). value = leaf nodes per second."""
    import torch

    import oracle as O
    import paper_2112_14944_gb300 as P
    import synth
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    g = synth.chung_lu(2_000_000, 10, 2.5, seed=0)
    k = 25
    ctx = P.Context(local_rank, torch_stream=True)
    stream = ctx._stream
    G = ctx.upload_graph(g)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    ms, res, clocks = _timed_steps(args, stream, flush, lambda: ctx.louvain_plus(G, k, with_info=True))
    launches = ctx.stats()["kernel_launches"]
    levels, info = res
    total = max_over_ranks(sum(ms), dev)
    ctx.profile(1)
    ctx.louvain_plus(G, k)
    ktimes = ctx.kernel_times()
    ctx.profile(False)
    # end to end through the public API from host buffers: the CSR uploaded
    # (and validated) in every step, the parent arrays returned to the host
    e2e_ms = []
    for _ in range(max(1, min(args.steps, 3))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Gh = ctx.upload_graph(g)
        ctx.louvain_plus(Gh, k)
        Gh.free()
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
    if rank != 0:
        return
    hbm, _, peak_kind = peaks()
    per = total / args.steps
    sizes = [g.n] + [int(p.max()) + 1 for p in levels]
    deg = np.diff(g.row_ptr)
    part = O.louvain_leaf_groups(g.n, levels)[0]
    src = np.repeat(np.arange(g.n), deg)
    same = part[src] == part[g.col]
    inside = np.bincount(part[src][same], minlength=sizes[1])
    dsum = np.bincount(part, weights=deg, minlength=sizes[1])
    Q1 = float(np.sum(inside / g.nnz - (dsum / g.nnz) ** 2))
    h_ms, h_n, _ = ktimes["hier"]
    # algorithmic bytes of the merge rounds: per pair scanned for the gains,
    # twice (largest gain, then its smallest arg), the 12 B record and the
    # size and degree sum of both groups (24 B); per pair contracted its 12 B
    # record, its two mapped ids (8 B) and one key and count (12 B); per
    # table slot the compaction scan (12 B; it also clears what it emits);
    # per level node and round ~16 words of node state (64 B)
    alg = (72.0 * info["list_visits"] + 32.0 * info["pair_visits"] + 12.0 * info["slot_visits"]
           + 64.0 * info["node_visits"])
    ach = alg / (h_ms / 1e3) / 1e9 if h_ms else None
    roof = {"kernel": "Louvain+ merge rounds (k_lp_*): pair-table atomics, table scans, node passes",
            "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm if ach else None,
            "launches": h_n, "alg_bytes_per_step": alg,
            "alg_bytes_note": "72 B per pair scanned for the gains + 32 B per pair contracted + 12 B per table slot + 64 B per node visit",
            "device_ms_per_step": h_ms, "traffic": None,
            "peak_kind": f"{peak_kind} hbm_gbs (copy bandwidth), frac of {peak_kind}"}
    cpu = None
    errors = None
    if world == 1 and not args.no_cpu_baseline:
        # the oracle on a bounded sample: a 1,000-node graph of the same kind,
        # k = 25; the GPU's hierarchy of the same sample must be identical
        gs = synth.chung_lu(1000, 10, 2.5, seed=0)
        t0 = time.perf_counter()
        ref = O.louvain_plus(gs.n, gs.row_ptr, gs.col, k)
        dt = time.perf_counter() - t0
        got = ctx.louvain_plus(ctx.upload_graph(gs), k)
        errors = {"sample_hierarchy_identical": len(got) == len(ref) and all(
            np.array_equal(np.asarray(a, np.int64), np.asarray(b, np.int64)) for a, b in zip(got, ref)),
                  "sample_levels": [int(p.max()) + 1 for p in ref]}
        cpu = {"value": gs.n / dt, "unit": "leaf nodes/s", "cores": 1, "kind": "oracle",
               "sample": "the oracle's Louvain+ hierarchy (exact rational gains, plain Python) of a 1,000-node "
                         "Chung-Lu graph of the same kind, k = 25"}
    line = {
        "metric": "Louvain+ hierarchy of a 2M-node power-law graph (k = 25), leaf nodes per second",
        "value": g.n / (per / 1e3), "unit": "leaf nodes/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": per, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": HIER_WORKLOAD, "graph": "chung-lu", "n": g.n, "nnz": int(g.nnz), "mean_degree": 10,
                   "exponent": 2.5, "seed": 0, "k": k, "l2": "flushed between timed steps (512 MB write)",
                   "parallelism": f"replicas x{world}"},
        "levels": sizes, "rounds": info["rounds"], "level1_modularity": Q1,
        "isolated_leaves": int((deg == 0).sum()),
        "errors": errors, "roofline": roof,
        "e2e": {"value": g.n / (float(np.median(e2e_ms)) / 1e3), "unit": "leaf nodes/s",
                "h2d_bytes_per_step": int(g.row_ptr.nbytes + g.col.nbytes),
                "d2h_bytes_per_step": int(4 * sum(sizes[:-1])), "ms_per_step": float(np.median(e2e_ms))},
        "cpu_baseline": cpu, "gpu_launches": int(launches * args.steps), "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- view of a 2M-node graph
VIEW2M_WORKLOAD = "chung_lu_n2000000_deg10_view8192"


def run_view2m(args, rank, world, local_rank):
    """The differentiable-layout workload: Chung-Lu n = 2,000,000, mean degree
    10, exponent 2.5, seed 0; a view of 8,192 nodes drawn uniformly (seed 0).
    One step = graph ingest + validation, FP32 DPPR / PDist among the view
    (n_clamp = n) with the FP64 certificate, then the stress energy of a layout
    of the view and its gradient through the autograd function (forward + the
    hand-written backward, pair recomputation)."""
    import torch

    import paper_2112_14944_gb300 as P
    import synth
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    g = synth.chung_lu(2_000_000, 10, 2.5, seed=0)
    k = 8192
    view_h = synth.sample_view(g.n, k, seed=0)
    ctx = P.Context(local_rank, torch_stream=True)
    stream = ctx._stream
    rp = torch.from_numpy(g.row_ptr).to(dev)
    col = torch.from_numpy(g.col).to(dev)
    view = torch.from_numpy(view_h).to(dev)
    D = torch.empty((k, k), dtype=torch.float32, device=dev)
    Dl = torch.empty_like(D)
    X0 = torch.from_numpy(synth.uniform_x0(k, seed=0) * 8.0).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    SE = P.StressEnergy

    def step():
        G = ctx.upload(g.n, rp, col)
        launches = ctx.stats()["kernel_launches"]
        _, _, cert, status = ctx.dppr(G, view, ALPHA, EPS, P.FP32, dppr_out=D, pdist_out=Dl, cert=True)
        sd = ctx.stats()
        launches += sd["kernel_launches"]
        X = X0.clone().requires_grad_(True)
        with torch.cuda.stream(stream):
            e = SE.apply(X, Dl, ctx)
            launches += ctx.stats()["kernel_launches"]
            e.backward()
            launches += ctx.stats()["kernel_launches"]
        G.free()
        return sd, status, float(cert.max()), launches, X.grad

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier_if_group()
    torch.cuda.synchronize()
    ctx.profile(PROF_EVERY)
    sampler = ClockSampler(local_rank)
    sampler.start()
    ms, sts, certs, launches, bytes_sweep, sweeps = [], [], [], 0, 0.0, 0
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sd, st, cm, nl, gx = step()
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
        sts.append(st)
        certs.append(cm)
        launches += nl
        bytes_sweep += sd["bytes_sweep"]
        sweeps += sd["sweeps_main"] + sd["sweeps_refine"]
    torch.cuda.synchronize()
    sampler.stop()
    ktimes = ctx.kernel_times()
    ctx.profile(False)
    assert all(x == 0 for x in sts) and max(certs) <= EPS, (sts, max(certs))
    assert bool(torch.isfinite(gx).all())
    total = max_over_ranks(sum(ms), dev)
    # Algorithm 2's frontier on this workload: per power-iteration sweep, the
    # share of (node, source) entries whose push residue is above GFP's
    # threshold for eps (512 of the view's sources; outside the timed steps)
    nf, T = 512, 140
    G = ctx.upload(g.n, rp, col)
    act = ctx.frontier_profile(G, view_h[:nf].copy(), T, ALPHA, EPS)
    G.free()
    frac = act / float(g.n * nf)
    frontier = {"sources": nf, "sweeps": T, "active_fraction_every_10_sweeps": [float(x) for x in frac[::10]],
                "max_active_fraction": float(frac.max()), "argmax_sweep": int(frac.argmax()),
                "mean_active_fraction_first_third": float(frac[:T // 3].mean()),
                "sweeps_with_any_active": int((act > 0).sum())}
    if rank != 0:
        return
    hbm, _, peak_kind = peaks()
    sw_ms, sw_all, sw_n = ktimes["sweep"]
    per = bytes_sweep / max(1, sw_all)
    ach = per / (sw_ms / max(1, sw_n) / 1e3) / 1e9 if sw_n else None
    roof = {"kernel": "propagation sweep (k_sweep): the [2M][G] state streams from HBM", "bound": "hbm",
            "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm if ach else None,
            "launches": sw_all, "timed_launches": sw_n, "avg_launch_us": 1e3 * sw_ms / max(1, sw_n),
            "alg_bytes_per_launch": per, "traffic": None,
            "peak_kind": f"{peak_kind} hbm_gbs (copy bandwidth), frac of {peak_kind}"}
    entries = float(k) * k
    line = {
        "metric": "DPPR entries/s, 8,192-node view of a 2M-node Chung-Lu graph (+ energy and backward)",
        "value": whole_job_rate(entries, args.steps, world, total), "unit": "entries/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": VIEW2M_WORKLOAD, "graph": "chung-lu", "n": g.n, "nnz": int(g.nnz), "mean_degree": 10,
                   "exponent": 2.5, "seed": 0, "view": "8,192 nodes uniform without replacement (seed 0)",
                   "n_clamp": g.n, "alpha": ALPHA, "eps": EPS,
                   "propagation": "fp32 chebyshev + fp64 residual certificate + fp32 refinement",
                   "energy": "stress energy of U[-8,8]^2 coordinates + backward (autograd.Function)",
                   "l2": "flushed between timed steps (512 MB write)", "parallelism": f"replicas x{world}"},
        "sweeps_per_step": sweeps / args.steps, "max_cert": max(certs), "roofline": roof,
        "frontier": frontier,
        "kernel_share": class_share(ktimes, args.steps), "gpu_launches": int(launches), "clocks": sampler.summary(),
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- small FP64 workload
SMALL_WORKLOAD = "chung_lu_n1000_deg10_fp64"


def run_small(args, rank, world, local_rank):
    """The small FP64 workload: Chung-Lu n = 1,000, mean degree 10, exponent
    2.5, seed 0; all-pairs FP64 DPPR -> PDist -> 300 FP64 layout updates from
    U[-1,1]^2 (seed 0); device buffers. Reported as latency (it fits in L2)."""
    import torch

    import paper_2112_14944_gb300 as P
    import synth
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    n = 1000
    g = synth.chung_lu(n, 10, 2.5, seed=0)
    ctx = P.Context(local_rank, torch_stream=True)
    stream = ctx._stream
    rp = torch.from_numpy(g.row_ptr).to(dev)
    col = torch.from_numpy(g.col).to(dev)
    view = torch.arange(n, dtype=torch.int32, device=dev)
    D = torch.empty((n, n), dtype=torch.float64, device=dev)
    Dl = torch.empty_like(D)
    x0 = torch.from_numpy(synth.uniform_x0(n, seed=0).astype(np.float64)).to(dev)
    xo = torch.empty_like(x0)

    def step():
        G = ctx.upload(n, rp, col)
        launches = ctx.stats()["kernel_launches"]
        _, _, cert, status = ctx.dppr(G, view, ALPHA, EPS, P.FP64, dppr_out=D, pdist_out=Dl, cert=True, out64=True)
        launches += ctx.stats()["kernel_launches"]
        _, s = ctx.layout(Dl, x0, 300, P.FP64, x_out=xo, stress=True)
        launches += ctx.stats()["kernel_launches"]
        G.free()
        return status, float(cert.max()), launches, s

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ms, sts, certs, launches = [], [], [], 0
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st, cm, nl, s = step()
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
        sts.append(st)
        certs.append(cm)
        launches += nl
    assert all(x == 0 for x in sts) and max(certs) <= EPS
    total = max_over_ranks(sum(ms), dev)
    if rank != 0:
        return
    line = {
        "metric": "DPPR entries/s, Chung-Lu n=1k, FP64 plain method (DPPR + PDist + 300 layout updates)",
        "value": whole_job_rate(float(n) * n, args.steps, world, total), "unit": "entries/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": SMALL_WORKLOAD, "graph": "chung-lu", "n": n, "mean_degree": 10, "exponent": 2.5,
                   "seed": 0, "alpha": ALPHA, "eps": EPS, "layout_iters": 300,
                   "l2": "not flushed: the whole workload fits in L2 (reported as latency)",
                   "parallelism": f"replicas x{world}"},
        "final_stress": s, "max_cert": max(certs), "gpu_launches": int(launches),
        "layout_iters_per_s": 300 / (total / args.steps / 1e3),
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- our arm
def run_ours(args, rank, world, local_rank):
    import torch

    import paper_2112_14944_gb300 as P
    import synth

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    n = args.n
    g = synth.chung_lu(n, args.deg, 2.5, seed=0)
    x0_h = synth.uniform_x0(n, seed=0)
    ctx = P.Context(local_rank, torch_stream=True)
    stream = ctx._stream
    rp = torch.from_numpy(g.row_ptr).to(dev)
    col = torch.from_numpy(g.col).to(dev)
    view = torch.arange(n, dtype=torch.int32, device=dev)
    D = torch.empty((n, n), dtype=torch.float32, device=dev)
    Dl = torch.empty((n, n), dtype=torch.float32, device=dev)
    x0 = torch.from_numpy(x0_h).to(dev)
    xo = torch.empty_like(x0)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    torch.cuda.synchronize()

    def step(rec=None):
        if rec is not None:
            rec[0].record(stream)
        G = ctx.upload(n, rp, col)
        st = ctx.stats()
        launches = st["kernel_launches"]
        _, _, cert, status = ctx.dppr(G, view, ALPHA, EPS, P.FP32, dppr_out=D, pdist_out=Dl, cert=True)
        sd = ctx.stats()
        launches += sd["kernel_launches"]
        if rec is not None:
            rec[1].record(stream)
        _, s = ctx.layout(Dl, x0, args.iters, P.FP32, x_out=xo, stress=True)
        sl = ctx.stats()
        launches += sl["kernel_launches"]
        if rec is not None:
            rec[2].record(stream)
        G.free()
        return launches, sd, sl, s, status, cert

    for _ in range(args.warmup):
        flush.zero_()
        _, _, _, _, status, cert = step()
        assert status == 0 and cert.max() <= EPS, (status, cert.max())
    torch.cuda.synchronize()
    barrier_if_group()
    torch.cuda.synchronize()
    ctx.profile(PROF_EVERY)
    sampler = ClockSampler(local_rank)
    sampler.start()
    step_ms, dppr_ms, layout_ms = [], [], []
    launches = 0
    bytes_sweep = bytes_ly = bytes_apply = flops_factor = 0.0
    sweeps = 0
    statuses, certs = [], []
    wall0 = time.perf_counter()
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()  # outside the step's events
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        nl, sd, sl, stress, status, last_cert = step(ev)
        statuses.append(status)
        certs.append(float(last_cert.max()))
        launches += nl
        bytes_sweep += sd["bytes_sweep"]
        sweeps += sd["sweeps_main"] + sd["sweeps_refine"]
        bytes_ly += sl["bytes_ly"]
        bytes_apply += sl["bytes_apply"]
        flops_factor += sl["flops_factor"]
        ev[2].synchronize()
        dppr_ms.append(ev[0].elapsed_time(ev[1]))
        layout_ms.append(ev[1].elapsed_time(ev[2]))
        step_ms.append(ev[0].elapsed_time(ev[2]))
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    barrier_if_group()
    torch.cuda.synchronize()
    sampler.stop()
    ktimes = ctx.kernel_times()
    ctx.profile(False)
    # every timed step converged and is certified within eps (checked after the clock)
    assert all(st == 0 for st in statuses) and max(certs) <= EPS, (statuses, max(certs))
    total_ms = sum(step_ms)
    total_ms = max_over_ranks(total_ms, dev)
    entries = float(n) * n
    value = whole_job_rate(entries, args.steps, world, total_ms)

    # ---- end to end through the public API with pinned host buffers
    e2e = None
    if args.e2e_steps > 0:
        pin = lambda a: torch.from_numpy(a).pin_memory().numpy()  # noqa: E731
        rp_h, col_h, x0_p = pin(g.row_ptr), pin(g.col), pin(x0_h)
        view_h = pin(np.arange(n, dtype=np.int32))
        D_h = torch.empty((n, n), dtype=torch.float32).pin_memory().numpy()
        Dl_h = torch.empty((n, n), dtype=torch.float32).pin_memory().numpy()
        X_h = torch.empty((n, 2), dtype=torch.float32).pin_memory().numpy()
        e2e_ms, e2e_st, e2e_cert = [], [], []
        for _ in range(args.e2e_steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            G = ctx.upload(n, rp_h, col_h)
            _, _, cert_h, st_h = ctx.dppr(G, view_h, ALPHA, EPS, P.FP32, dppr_out=D_h, pdist_out=Dl_h, cert=True)
            ctx.layout(Dl_h, x0_p, args.iters, P.FP32, x_out=X_h, stress=True)
            G.free()
            e2e_ms.append(1e3 * (time.perf_counter() - t0))
            e2e_st.append(st_h)
            e2e_cert.append(float(cert_h.max()))
        assert all(st == 0 for st in e2e_st) and max(e2e_cert) <= EPS, (e2e_st, max(e2e_cert))
        tot = sum(e2e_ms)
        tot = max_over_ranks(tot, dev)
        h2d = rp_h.nbytes + col_h.nbytes + view_h.nbytes + Dl_h.nbytes + x0_p.nbytes
        d2h = D_h.nbytes + Dl_h.nbytes + X_h.nbytes + 8 * n
        e2e = {"value": whole_job_rate(entries, args.e2e_steps, world, tot), "unit": "entries/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "ms_per_step": tot / args.e2e_steps, "max_cert": max(e2e_cert)}

    # ---- the plain FP64 GPU path on the same workload and eps: FP64 power
    # iteration (PPRVIZ_FP64) and the FP64 layout, device buffers, one step
    fp64 = None
    if args.fp64_steps > 0:
        D64 = torch.empty((n, n), dtype=torch.float64, device=dev)
        Dl64 = torch.empty((n, n), dtype=torch.float64, device=dev)
        x64 = x0.double()
        xo64 = torch.empty_like(x64)

        def step64():
            G = ctx.upload(n, rp, col)
            _, _, c64, st64 = ctx.dppr(G, view, ALPHA, EPS, P.FP64, dppr_out=D64, pdist_out=Dl64, cert=True,
                                       out64=True)
            ctx.layout(Dl64, x64, args.iters, P.FP64, x_out=xo64, stress=True)
            G.free()
            return st64, float(c64.max())

        step64()  # warm-up (workspace, first-use allocations)
        ms64, st64s, c64s = [], [], []
        for _ in range(args.fp64_steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st64, c64 = step64()
            e1.record(stream)
            e1.synchronize()
            ms64.append(e0.elapsed_time(e1))
            st64s.append(st64)
            c64s.append(c64)
        assert all(st == 0 for st in st64s) and max(c64s) <= EPS, (st64s, max(c64s))
        t64 = max_over_ranks(sum(ms64), dev) / len(ms64)
        fp64 = {"value": whole_job_rate(entries, 1, world, t64), "unit": "entries/s", "ms_per_step": t64,
                "steps": len(ms64), "max_cert": max(c64s), "speedup_of_fp32_step": t64 / (total_ms / args.steps),
                "path": "FP64 power iteration (a-priori sweep count) + FP64 residual certificate; FP64 PDist; "
                        "FP64 L^w inverse and layout passes; same graph, view, eps, iterations"}
        del D64, Dl64

    if rank != 0:
        return
    hbm, sm_max, peak_kind = peaks()
    names = {"sweep": ("propagation sweep (k_sweep)", bytes_sweep),
             "ly": ("all-pairs L^Y pass (k_sympass_pipe<0>, persistent, TMA tile pipeline)", bytes_ly),
             "apply": ("(L^w)^+ apply pass (k_sympass_pipe<1>, persistent, TMA tile pipeline)", bytes_apply)}
    kernels = {}
    # algorithmic bytes per launch = the class's bytes over all its launches in
    # the timed steps / those launches; achieved = that / the average duration
    # of its timed launches
    for cls, (label, alg) in names.items():
        ms, cnt, timed = ktimes[cls]
        if timed == 0 or ms <= 0:
            continue
        per = alg / cnt
        ach = per / (ms / timed / 1e3) / 1e9
        kernels[cls] = {"kernel": label, "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                        "frac": ach / hbm, "launches": cnt, "timed_launches": timed,
                        "avg_launch_us": 1e3 * ms / timed, "alg_bytes_per_launch": per,
                        "traffic": measured_traffic(cls)}
    ms, cnt, timed = ktimes["factor"]
    if timed and ms > 0 and flops_factor > 0:
        tf32, tf_kind = tf32_tflops()
        per = flops_factor / cnt
        ach = per / (ms / timed / 1e3) / 1e12
        kernels["factor"] = {"kernel": "L^w build + inverse: symmetric block sweep with lookahead (k_fac_*); "
                                       "trailing update on tcgen05.mma kind::tf32 (3xTF32)",
                             "bound": "tensor", "achieved": ach, "peak": tf32, "unit": "TFLOP/s",
                             "frac": ach / tf32, "issued_frac_3xtf32": 3 * ach / tf32,
                             "launches": cnt, "timed_launches": timed,
                             "avg_launch_us": 1e3 * ms / timed, "alg_flops_per_launch": per,
                             "traffic": measured_traffic("factor"), "peak_kind": tf_kind}
    share = class_share(ktimes, args.steps)
    dom = max(kernels, key=lambda c: share[c]["ms"]) if kernels else None
    roof = dict(kernels[dom]) if dom else None
    if roof is not None and roof["bound"] == "hbm":
        roof["peak_kind"] = f"{peak_kind} hbm_gbs (copy bandwidth), frac of {peak_kind}"
    cpu, errors = None, None
    if world == 1 and not args.no_cpu_baseline:
        e, t = cpu_oracle_sample(g, 16)
        cpu = {"value": e / t, "unit": "entries/s", "cores": 1, "kind": "oracle",
               "sample": "16 seeded sources: FP64 DPPR rows + PDist rows by power iteration (scipy sparse, 1 thread)"}
        if args.cpu_all_cores:
            ea, ta, cores = cpu_oracle_all_cores(g, 16)
            cpu["all_cores"] = {"value": ea / ta, "unit": "entries/s", "cores": cores,
                                "sample": f"{cores} x 16 seeded sources, one spawned process per core"}
        # per-result error of the last timed step's outputs against the oracle's rows
        src = synth.sample_view(n, 16, seed=1)
        errors = oracle_errors(g, src, D[torch.from_numpy(src).to(dev).long()].cpu().numpy(),
                               Dl[torch.from_numpy(src).to(dev).long()].cpu().numpy(), last_cert)
        # one layout update from X0 on the step's PDist: error bound of the exact update
        x1 = torch.empty_like(x0)
        ctx.layout(Dl, x0, 1, P.FP32, x_out=x1, stress=False)
        bnd, jac = layout_update_error_bound(Dl.cpu().numpy(), x0_h, x1.cpu().numpy())
        errors["layout_one_update_err_bound"] = bnd
        errors["layout_one_update_err_jacobi_estimate"] = jac
        errors["max_cert_timed_steps"] = max(certs)
    line = {
        "metric": "DPPR entries/s at n=10k, err<=1e-6 vs FP64; layout iters/s; % HBM roofline",
        "value": value, "unit": "entries/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": config(args, world),
        "phases": {"dppr_pdist_ms": statistics.mean(dppr_ms), "layout_ms": statistics.mean(layout_ms),
                   "dppr_entries_per_s_phase": entries / (statistics.mean(dppr_ms) / 1e3),
                   "layout_iters_per_s": args.iters / (statistics.mean(layout_ms) / 1e3),
                   "sweeps_per_step": sweeps / args.steps, "final_stress": stress,
                   "wall_s_timed_region": wall},
        "roofline": roof, "roofline_kernels": kernels, "kernel_share": share,
        "kernel_share_note": "per class and step: the mean CUDA-event duration of the class's timed launches "
                             "times all its launches; classes overlap (the inverse's lookahead stream, "
                             "programmatic dependent launches of the row reduces), so the sum exceeds the step",
        "gpu_launches": int(launches), "errors": errors, "vs_fp64_gpu": fp64,
        "e2e": e2e, "cpu_baseline": cpu, "clocks": sampler.summary(),
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.n is None:
        args.n = 20000 if args.workload == "dense" else 10000
    if args.case:
        run_case(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1 and args.impl == "ours":
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload == "dense":
        run_dense(args, rank, world, local_rank)
    elif args.workload == "views":
        run_views(args, rank, world, local_rank)
    elif args.workload == "taupush":
        run_taupush(args, rank, world, local_rank)
    elif args.workload == "level":
        run_level(args, rank, world, local_rank)
    elif args.workload == "directed":
        run_directed(args, rank, world, local_rank)
    elif args.workload == "metrics":
        run_metrics(args, rank, world, local_rank)
    elif args.workload == "hierarchy":
        run_hierarchy(args, rank, world, local_rank)
    elif args.workload == "view2m":
        run_view2m(args, rank, world, local_rank)
    elif args.workload == "small":
        run_small(args, rank, world, local_rank)
    else:
        run_ours(args, rank, world, local_rank)
    if world > 1 and args.impl == "ours":
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
