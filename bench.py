"""Benchmark: LeanVec search QPS at 10-recall@10 = 0.90 on one GB300 (per rank).

Workload (default): 1M x 768 anisotropic Gaussian mixture (1000 components, i^-1
spectrum, unit-normalised, inner product), 10k in-distribution queries; LeanVec-ID
d = 160 (second moments + FP64 eigh on a 100k subsample), LVQ-8 primary + LVQ-8
secondary, GPU-built graph R = 64, L_build = 128.  A step is one pass of the
search path (projection A q -> beam search over primaries -> rerank with
secondaries -> top-10) over the 10k queries, inputs resident in HBM; the beam width
L (rerank = L) is the smallest of a sweep whose recall@10 reaches 0.90.

Reported next to it: the same metric end to end through the C ABI with host
buffers (e2e), the plain full-dimensional float32 graph search on the same graph
(baseline_fp32, its own L for 0.90), the beam kernel's HBM roofline fraction, and
the CPU oracle timed on a bounded query sample on this host (cpu_baseline).

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]
N > 1 runs N independent replicas (one per GPU, weak scaling, no collective on the
data path; a barrier and a max-reduction of the timings only).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

L_GRID = [10, 12, 16, 20, 24, 28, 32, 36, 40, 44, 48, 52, 56, 60, 64, 72, 80, 88, 96, 104, 112, 120, 128, 132, 136,
          140, 144, 148, 152, 156, 160, 176, 200, 256, 320, 384, 448, 512]

# DRAM bytes (read + write) of the search kernels of one search, from one ncu capture of the same
# configuration (dram__bytes_read.sum + dram__bytes_write.sum), valid only for the kernel sources
# it was taken on (the sha1 of beam.cuh, search_lvq8.cu and rerank.cu, and since the visited cache
# of 16-bit tags also of search_launch.cuh and search_lvq8_tags.cu) and the visited-cache slot width.
TRAFFIC_RECORDS = [
    # beam_kernel (3.067 GB read + 10.7 MB written) + rerank_kernel (1.198 GB + 0.15 MB) of one search
    {"src_sha1": "9fb2aadd90f9d3ae629c84c792cada92736d15aa", "n": 1_000_000, "m": 10_000, "L": 160, "width": 2, "hash": 0,
     "projection": "bf16", "alpha": 1.0, "rule": 0, "bytes": 3066597888 + 10704640 + 1198200320 + 154624},
    # the default graph (unit-L2 rule, alpha 1.02) at its L for 0.90: beam 3.271 GB + 10.2 MB, rerank 1.107 GB + 0.25 MB
    {"src_sha1": "9fb2aadd90f9d3ae629c84c792cada92736d15aa", "n": 1_000_000, "m": 10_000, "L": 148, "width": 2, "hash": 0,
     "projection": "bf16", "alpha": 1.02, "rule": 1, "bytes": 3271060992 + 10185216 + 1106905856 + 252160},
    # the same rule on a graph built on full-D LVQ-8 codes, L = 120: beam 2.733 GB + 8.8 MB, rerank 0.893 GB + 1.2 MB
    {"src_sha1": "9ea3355bc525640bcd5ba8c54cfb9beac141d1aa", "n": 1_000_000, "m": 10_000, "L": 120, "width": 2, "hash": 0, "projection": "bf16",
     "alpha": 1.02, "rule": 1, "graph": "full", "bytes": 2733314560 + 8754688 + 893092608 + 1217024},
    # that graph with the expansion budget max_hops = L, L = 128, one launch each: beam 2.455 GB + 8.3 MB,
    # rerank 0.954 GB + 1.2 MB
    {"src_sha1": "9ea3355bc525640bcd5ba8c54cfb9beac141d1aa", "n": 1_000_000, "m": 10_000, "L": 128, "max_hops": 128,
     "width": 2, "hash": 0, "projection": "bf16", "alpha": 1.02, "rule": 1, "graph": "full",
     "bytes": 2454921216 + 8330752 + 954114560 + 1157888},
    # the default: the same, 7296 + 2704 queries as two sub-batches on two streams (four launches):
    # beam 1.698 GB + 0.508 GB read, rerank 0.688 GB + 0.255 GB read, 9.8 MB written in all
    {"src_sha1": "d570e3e1d2fda9ca3c092fe3121669cb1dd17e74", "n": 1_000_000, "m": 10_000, "L": 128, "max_hops": 128,
     "width": 2, "hash": 0, "projection": "bf16", "alpha": 1.02, "rule": 1, "graph": "full",
     "bytes": 3148564224 + 9814016},
    # the same after the score-first beam-position search (same loads): 3.147 GB read, 9.9 MB written
    {"src_sha1": "5cd3a18943e7fa552c926df8ed848773dac7f10e", "n": 1_000_000, "m": 10_000, "L": 128, "max_hops": 128,
     "width": 2, "hash": 0, "projection": "bf16", "alpha": 1.02, "rule": 1, "graph": "full",
     "bytes": 3147171584 + 9867776},
    # the same with the query constants computed in the scorers (no kernel of their own): 3.144 GB
    # read, 8.1 MB written
    {"src_sha1": "adabdf5c923b6df5930577829fe01484d40bee83", "n": 1_000_000, "m": 10_000, "L": 128, "max_hops": 128,
     "width": 2, "hash": 0, "projection": "bf16", "alpha": 1.02, "rule": 1, "graph": "full",
     "bytes": 3144495360 + 8056832},
    # the calibrated budget, hop factor 0.5 (L = 152, max_hops = 76): beam 0.962 + 0.371 GB read,
    # rerank 0.779 + 0.344 GB read, 3.8 MB written
    {"src_sha1": "adabdf5c923b6df5930577829fe01484d40bee83", "n": 1_000_000, "m": 10_000, "L": 152, "max_hops": 76,
     "width": 2, "hash": 0, "projection": "bf16", "alpha": 1.02, "rule": 1, "graph": "full",
     "bytes": 2459870720},
    # hop factor 0.6 (L = 140, max_hops = 84)
    {"src_sha1": "adabdf5c923b6df5930577829fe01484d40bee83", "n": 1_000_000, "m": 10_000, "L": 140, "max_hops": 84,
     "width": 2, "hash": 0, "projection": "bf16", "alpha": 1.02, "rule": 1, "graph": "full",
     "bytes": 2505062656},
    # records prefetched into L2 at the visited test, L = 152, max_hops = 76: beam 0.865 + 0.366 GB
    # read, rerank 0.778 + 0.344 GB read, 6.8 MB written (mean of the two profiled searches)
    {"src_sha1": "9c0aada7abc74f8df81a778ce8e0f6cdc14a6801", "n": 1_000_000, "m": 10_000, "L": 152, "max_hops": 76,
     "width": 2, "hash": 0, "projection": "bf16", "alpha": 1.02, "rule": 1, "graph": "full",
     "bytes": 2361016064},
    # the same kernel after the search launchers moved into search_launch.cuh (visited cache of
    # 32-bit ids, the default): beam 2.465 GB read, rerank 2.246 GB read, 13.7 MB written (two searches)
    {"src_sha1": "1a2d083cdc2fc77fbe3145b0f3ead1ea2711fa9f", "n": 1_000_000, "m": 10_000, "L": 152, "max_hops": 76,
     "width": 2, "hash": 0, "projection": "bf16", "alpha": 1.02, "rule": 1, "graph": "full", "vbits": 32,
     "bytes": 2362186752},
    # the visited cache of 16-bit tags (--visited-bits 16): beam 2.367 GB read, rerank 2.246 GB read,
    # 12.7 MB written (two searches)
    {"src_sha1": "1a2d083cdc2fc77fbe3145b0f3ead1ea2711fa9f", "n": 1_000_000, "m": 10_000, "L": 152, "max_hops": 76,
     "width": 2, "hash": 0, "projection": "bf16", "alpha": 1.02, "rule": 1, "graph": "full", "vbits": 16,
     "bytes": 2312933760},
]


def beam_src_sha1() -> str:
    import hashlib
    root = os.path.join(ROOT, "paper_2312_16335_gb300", "csrc")
    h = hashlib.sha1()
    for f in ("beam.cuh", "search_lvq8.cu", "rerank.cu", "search_launch.cuh", "search_lvq8_tags.cu"):
        h.update(open(os.path.join(root, f), "rb").read())
    return h.hexdigest()


def recorded_traffic(args, L, max_hops=0):
    sha = beam_src_sha1()
    for r in TRAFFIC_RECORDS:
        if (r["src_sha1"] == sha and r["n"] == args.n and r["m"] == args.m and r["L"] == L and
                r.get("max_hops", 0) == max_hops and
                r["width"] == args.width and r["hash"] == args.hash and r["projection"] == args.projection and
                r.get("alpha") == args.alpha and r.get("rule") == args.rule and
                r.get("graph", "primary") == getattr(args, "graph", "primary") and
                r.get("secondary", "lvq8") == getattr(args, "secondary", "lvq8") and
                r.get("vbits", 32) == (getattr(args, "vbits", 0) or 32)):
            return r["bytes"]
    return None
TARGET = 0.90


def log(*a):
    if int(os.environ.get("RANK", "0")) == 0:
        print("[bench]", *a, file=sys.stderr, flush=True)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        j = json.load(open(p))
        return float(j["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.3)
        except FileNotFoundError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait(timeout=5)

    def summary(self):
        mhz, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                mhz.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(mhz) if mhz else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(mhz)}


def ground_truth(X: torch.Tensor, Q: torch.Tensor, k: int = 10, chunk: int = 131072, l2: bool = False) -> torch.Tensor:
    """Exact top-k inner products, or with l2 the k nearest in Euclidean distance (largest
    2 <q, x> - ||x||^2); float32 on the GPU, TF32 off."""
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    best_s = torch.full((Q.shape[0], k), -float("inf"), device=Q.device)
    best_i = torch.full((Q.shape[0], k), -1, dtype=torch.int64, device=Q.device)
    for s in range(0, X.shape[0], chunk):
        S = Q @ X[s:s + chunk].T
        if l2:
            S = 2 * S - (X[s:s + chunk].double() ** 2).sum(1).float()[None, :]
        v, i = torch.topk(S, k, dim=1)
        cs = torch.cat([best_s, v], 1)
        ci = torch.cat([best_i, i + s], 1)
        o = torch.topk(cs, k, dim=1)
        best_s, best_i = o.values, torch.gather(ci, 1, o.indices)
    torch.backends.cuda.matmul.allow_tf32 = prev
    return best_i


def recall_at(ids: torch.Tensor, truth: torch.Tensor, k: int = 10) -> float:
    a = ids[:, :k].long()
    hit = (a.unsqueeze(2) == truth[:, :k].unsqueeze(1)).any(dim=2) & (a >= 0)
    return float(hit.float().sum().item()) / (k * ids.shape[0])


def calibrate(search_fn, truth, k):
    """Smallest L of the grid with recall@k >= 0.90; the (L, recall) trace."""
    trace = []
    chosen = None
    for L in L_GRID:
        ids = search_fn(L)
        r = recall_at(ids, truth, k)
        trace.append((L, r))
        if r >= TARGET:
            chosen = L
            break
    return chosen, trace


HOP_FACTORS = (0.0, 1.5, 1.33, 1.2, 1.1, 1.0, 0.9, 0.8, 0.7, 0.6, 0.5, 0.4)


def hop_limit(c, L):
    """The expansion budget max_hops = ceil(c L) of hop factor c (0: no limit)."""
    return 0 if not c else int(math.ceil(c * L - 1e-9))


def calibrate_budget(search_fn, time_fn, truth, k, factors=HOP_FACTORS):
    """Early termination by an expansion budget (the query descriptor's max_hops): for each hop
    factor c, the smallest grid L with recall@k >= 0.90 under max_hops = ceil(c L), timed; returns
    (L, max_hops, recall, table) of the fastest.  search_fn(L, mh) -> ids; time_fn(L, mh) -> QPS."""
    table = []
    for c in factors:
        L, trace = calibrate(lambda L: search_fn(L, hop_limit(c, L)), truth, k)
        if L is None:
            table.append({"hop_factor": c, "L": None, "recall_trace": trace[-2:]})
            continue
        mh = hop_limit(c, L)
        row = {"hop_factor": c, "L": L, "max_hops": mh, "recall": dict(trace)[L], "qps": time_fn(L, mh),
               "recall_trace": trace[-2:]}
        # QPS at recall 0.90 by log-linear interpolation between the bracketing grid points (the
        # grid point below 0.90 timed as well); the reported value stays the grid point's
        row["qps_interpolated"] = row["qps"]
        if len(trace) >= 2:
            (L0, r0), (L1, r1) = trace[-2], trace[-1]
            q0 = time_fn(L0, hop_limit(c, L0))
            row["qps_below"] = q0
            if r1 > r0:
                f = (TARGET - r0) / (r1 - r0)
                row["qps_interpolated"] = math.exp(math.log(q0) + f * (math.log(row["qps"]) - math.log(q0)))
        table.append(row)
    ok = [t for t in table if t.get("qps")]
    if not ok:
        return None, 0, None, table
    best = max(ok, key=lambda t: t["qps"])
    return best["L"], best["max_hops"], best["recall"], table


def qps_of(fn, m):
    """QPS of search fn(L, mh) over 5 timed calls after 2 untimed ones."""
    def q(L, mh):
        ms, _ = time_steps(lambda ev: fn(L, mh), 5, 2)
        return m * 5 / (ms / 1e3)
    return q


def choose_config(args, S, proj, k=10):
    """The id workload's LeanVec search configuration: --L/--max-hops when given, else the fastest
    (L, max_hops) of the hop-budget calibration (recall@k >= 0.90).  Returns (L, mh, recall, table)."""
    idx, Q, A, truth = S["idx"], S["Q"], S["A"], S["truth"]

    def lv_search(L, mh):
        return idx.search(Q, A, k=k, L=L, rerank=L, max_hops=mh, width=args.width, hash_slots=args.hash, queries_per_warp=args.qpw, visited_bits=args.vbits,
                          projection=proj)

    if args.L:
        return args.L, args.max_hops, recall_at(lv_search(args.L, args.max_hops)[0], truth, k), []
    factors = HOP_FACTORS if args.hop_sweep else (args.hop_factor,)
    L, mh, rec, table = calibrate_budget(lambda L, mh: lv_search(L, mh)[0], qps_of(lv_search, Q.shape[0]), truth, k,
                                         factors)
    if L is None:
        L, mh = L_GRID[-1], 0
        rec = recall_at(lv_search(L, mh)[0], truth, k)
    return L, mh, rec, table


def best_hop_factor(table, default):
    """The hop factor of the fastest calibrated row (the chosen configuration)."""
    ok = [t for t in table if t.get("qps")]
    return max(ok, key=lambda t: t["qps"])["hop_factor"] if ok else default


def id_config(args, workload, n_queries, L, mh, hop_factor, inf):
    """The id workload's configuration, the same dict in both arms' lines: what is searched and how,
    no results."""
    return {"workload": workload, "n": args.n, "D": args.D, "d": args.d, "queries": n_queries, "k": 10, "L": L,
            "rerank": L, "max_hops": mh, "hop_factor": hop_factor, "R": args.R, "L_build": args.L_build,
            "alpha": args.alpha, "prune_rule": args.rule, "graph_built_on": args.graph, "secondary": args.secondary,
            "projection": args.projection, "hash_slots": args.hash or "default", "width": args.width,
            "queries_per_warp": args.qpw or 1, "visited_bits": args.vbits or "default",
            "l2": "inputs larger than L2 (index %.2f GB vs 126 MB L2)" %
                  ((inf["primary_stride"] + inf["secondary_stride"] + 4 * inf["R"]) * args.n / 1e9)}


def replica_throughput(total_ms, units_per_step, steps, device=None):
    """Whole-job throughput of N independent replicas (one per rank, no data exchange): every rank
    timed the same number of steps; the job lasts as long as the slowest rank (max over ranks) and
    processed N x steps x units.  Returns (units per second, the max time in ms)."""
    dist = torch.distributed
    world = dist.get_world_size() if dist.is_available() and dist.is_initialized() else 1
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total = float(t.item())
    return units_per_step * steps * world / (total / 1e3), total


def time_steps(fn, steps, warmup, events=None):
    """Run `warmup` untimed steps, then time `steps` steps with CUDA events on the current stream.
    Returns (total milliseconds of all timed steps, per-step kernel milliseconds when `events`)."""
    st = torch.cuda.current_stream()
    for _ in range(warmup):
        fn(None)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    kern = []
    e0.record(st)
    for _ in range(steps):
        if events is not None:
            pair = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            pair[0].record(st)
            pair[1].record(st)  # materialise the handles before the library records them
            kern.append(pair)
            fn(pair)
        else:
            fn(None)
    e1.record(st)
    torch.cuda.synchronize()
    total_ms = e0.elapsed_time(e1)
    kern_ms = [a.elapsed_time(b) for a, b in kern]
    return total_ms, kern_ms


def setup(args, dev, with_base=True):
    from paper_2312_16335_gb300 import build_lib
    build_lib.build()  # no-op when the in-tree library is up to date
    import paper_2312_16335_gb300 as lv
    t0 = time.time()
    torch.manual_seed(0)
    X, Q, _ = workloads.make_workload_torch("anisotropic", args.n, args.m, args.D, args.components, cfg=2, device=dev)
    torch.cuda.synchronize()
    log(f"data {tuple(X.shape)} queries {tuple(Q.shape)} in {time.time() - t0:.1f}s")
    t0 = time.time()
    sub = torch.from_numpy(workloads.subsample_rows(args.n, min(args.n, 100_000), cfg=2)).to(dev)
    A = lv.leanvec_fit_id(X.index_select(0, sub).contiguous(), args.d)
    torch.cuda.synchronize()
    t_fit = time.time() - t0
    t0 = time.time()
    idx = lv.Index(dev.index).encode(X, A, primary_bits=8,
                                     secondary_bits=16 if getattr(args, "secondary", "lvq8") == "fp16" else 8)
    torch.cuda.synchronize()
    t_enc = time.time() - t0
    t0 = time.time()
    if getattr(args, "graph", "primary") == "full":
        # the graph both searches share is built on the unreduced vectors (LVQ-8 codes of x, the
        # full-precision stand-in), as the paper's search comparisons use a full-precision graph
        gi = lv.Index(dev.index).set_primary(X, None, 8, args.D)
    else:
        gi = idx
    gi.build_graph(R=args.R, L_build=args.L_build, alpha=args.alpha, passes=2, batch=args.batch, rule=args.rule,
                   seed=workloads.SEED_GRAPH + 2)
    gi.sync_status()
    graph, entry = gi.get_graph()
    if gi is not idx:
        idx.set_graph(graph, entry)
        del gi
    torch.cuda.synchronize()
    t_build = time.time() - t0
    log(f"fit {t_fit:.2f}s encode {t_enc:.2f}s build {t_build:.2f}s ({getattr(args, 'graph', 'primary')} graph)")
    base = lv.Index(dev.index).encode_fp32(X).set_graph(graph, entry) if with_base else None
    t0 = time.time()
    truth = ground_truth(X, Q, 10)
    log(f"ground truth {time.time() - t0:.1f}s")
    return dict(lv=lv, X=X, Q=Q, A=A, idx=idx, base=base, graph=graph, entry=entry, truth=truth,
                t_fit=t_fit, t_enc=t_enc, t_build=t_build)


def oracle_prepare(S, projection="bf16"):
    """Host copies and the oracle's own LVQ stores of the same vectors and projection; the
    queries projected in FP64 from the operands the GPU's projection multiplies (bf16-rounded
    for the bf16 projection), so that the oracle walks the same beam."""
    import oracle
    from oracle import rounding
    X = S["X"].cpu().numpy()
    A32 = S["A"].cpu().numpy()
    A = A32.astype(np.float64)
    Y = (X.astype(np.float64) @ A.T).astype(np.float32)
    prim = oracle.lvq_encode(Y, oracle.mean_fp32(Y), 8)
    sec = oracle.lvq_encode(X, oracle.mean_fp32(X), 8)
    Q32 = S["Q"].cpu().numpy()
    return dict(prim=prim, sec=sec, g=S["graph"].cpu().numpy(), entry=S["entry"], Qh=Q32.astype(np.float64),
                qp=rounding.project(Q32, A32, projection), truth=S["truth"].cpu().numpy())


def method_bytes_per_query(D, d, bits, R, hops, scored, rerank):
    """Algorithmic bytes of one query of the search: the query (4 D), one graph row per expansion
    (4 R ids + a 4-byte degree), one primary record per scored node (d bits / 8 code bytes + 8 bytes
    of constants, rounded up to 32-byte sectors) and one secondary record per reranked candidate
    (D code bytes + 8 bytes of constants)."""
    prim = -(-(d * bits // 8 + 8) // 32) * 32
    return 4 * D + hops * (4 * R + 4) + scored * prim + rerank * (D + 8)


def cpu_oracle_sample(O, L, budget_s, nthreads=0, max_hops=0, width=1):
    """Time the CPU oracle (C, OpenMP over queries) on a bounded query sample, with the GPU
    search's L, rerank, expansion budget and width."""
    import oracle
    cores = nthreads or os.cpu_count()
    Qh = O["Qh"]
    m = 64
    while True:
        t0 = time.perf_counter()
        r = oracle.search(O["g"], O["entry"], O["qp"][:m], k=10, L=L, rerank=L, prim=O["prim"], sec=O["sec"],
                          qs=Qh[:m], nthreads=cores, max_hops=max_hops, width=width)
        dt = time.perf_counter() - t0
        if dt > budget_s / 4 or m >= Qh.shape[0]:
            break
        m = min(Qh.shape[0], int(m * max(2.0, budget_s / 2 / max(dt, 1e-3))))
    rec = oracle.recall(r["ids"], O["truth"][:m], 10)
    return {"value": m / dt, "unit": "queries/s", "cores": cores, "kind": "oracle",
            "sample": f"first {m} of {Qh.shape[0]} queries, same graph/projection, L = rerank = {L}, "
                      f"max_hops = {max_hops or 'none'}, width {width}, k = 10",
            "recall_at_10": rec, "seconds": dt, "scored_per_query": float(r["scored"].mean()),
            "hops_per_query": float(r["hops"].mean())}


def bench_ood(args, dev):
    """Shifted-query workload: 1M x 512 database, 10k OOD test + 10k learning queries, d = 128.
    ID PCA vs LeanVec-OOD (Frank-Wolfe, eigenvector search) primaries on the same graph; plus
    the timed pair-loss forward + backward (differentiation form) on 10k x 100k sample pairs."""
    from paper_2312_16335_gb300 import build_lib
    build_lib.build()
    import paper_2312_16335_gb300 as lv
    n, m, D, d = args.n, args.m, 512, 128
    X, Q, Ql = workloads.make_workload_torch("anisotropic", n, m, D, 1000, cfg=3, device=dev, ood=True, m_learn=m)
    sub = torch.from_numpy(workloads.subsample_rows(n, min(n, 100_000), cfg=3)).to(dev)
    Xs = X.index_select(0, sub).contiguous()
    truth = ground_truth(X, Q, 10)
    fits = {}
    t0 = time.time()
    P = lv.leanvec_fit_id(Xs, d)
    fits["id"] = (P, P, {"seconds": time.time() - t0})
    for name, meth in (("ood_fw", lv.FIT_FW), ("ood_es", lv.FIT_ES)):
        t0 = time.time()
        A, B, rep = lv.leanvec_fit_ood(Xs, Ql, d, method=meth)
        rep = {k: v for k, v in rep.items() if k != "loss_trace"}
        rep["seconds"] = time.time() - t0
        fits[name] = (A, B, rep)
    # the differentiation form's gradient optimiser: Adam on the hand-written pair loss over the
    # same 10k learning queries x 100k database samples, from LeanVec-ID, spectral-norm projection
    # after every step; the best iterate of its trace
    t0 = time.time()
    A, B, trace = lv.fit_ood_gradient(Xs, Ql, d, steps=args.grad_steps, lr=args.grad_lr, A0=P)
    torch.cuda.synchronize()
    fits["ood_grad"] = (A, B, {"seconds": time.time() - t0, "steps": args.grad_steps, "lr": args.grad_lr,
                               "optimiser": "Adam + spectral-norm projection, best iterate",
                               "loss_first": trace[0], "loss_best": min(trace), "loss_last": trace[-1],
                               "best_step": int(np.argmin(trace))})
    # every projection's loss f(A, B) / (n m) on the learning pairs (the pair loss forward)
    with torch.no_grad():
        for name, (A, B, rep) in fits.items():
            rep["pair_loss"] = float(lv.OODLoss.apply(A.contiguous(), B.contiguous(), Ql, Xs))
    # differentiation form: one forward + backward over 10k x 100k pairs (tf32x3 tensor cores)
    Ap = torch.nn.Parameter(fits["id"][0].clone())
    Bp = torch.nn.Parameter(fits["id"][1].clone())
    torch.cuda.synchronize()
    times = []
    for i in range(3):
        t0 = time.perf_counter()
        loss = lv.OODLoss.apply(Ap, Bp, Ql, Xs)
        loss.backward()
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    mm, nn_ = Ql.shape[0], Xs.shape[0]
    # executed tf32 flops: forward 3 x 2 m n D, backward 3 x 2 m n (D + 2 d) (R, then R X' and R^T Q')
    flops = 3 * 2 * mm * nn_ * D + 3 * 2 * mm * nn_ * (D + 2 * d)
    diff = {"seconds": min(times[1:]), "pairs": mm * nn_, "tflops": flops / min(times[1:]) / 1e12}
    # one graph (built on the ID primaries), primaries swapped per projection
    idx = lv.Index(dev.index).encode(X, fits["id"][1], 8, 8, precision=lv.PREC_BF16)
    idx.build_graph(R=args.R, L_build=args.L_build, alpha=args.alpha, passes=2, batch=args.batch, rule=args.rule,
                    seed=workloads.SEED_GRAPH + 3)
    graph, entry = idx.get_graph()
    res = {}
    for name, (A, B, rep) in fits.items():
        ix = lv.Index(dev.index).encode(X, B, 8, 8, precision=lv.PREC_BF16).set_graph(graph, entry)
        per_L = {}
        hf = args.hop_factor
        for L in (16, 32, 64, 128):
            ids = ix.search(Q, A, k=10, L=L, rerank=L, width=args.width, projection=lv.PREC_BF16)[0]
            per_L[L] = recall_at(ids, truth)
        L90, trace = calibrate(lambda L: ix.search(Q, A, k=10, L=L, rerank=L, max_hops=hop_limit(hf, L),
                                                    width=args.width, projection=lv.PREC_BF16)[0], truth, 10)
        qps = None
        if L90:
            ms, _ = time_steps(lambda ev: ix.search(Q, A, k=10, L=L90, rerank=L90, max_hops=hop_limit(hf, L90),
                                                    width=args.width, projection=lv.PREC_BF16), 10, 3)
            qps = Q.shape[0] * 10 / (ms / 1e3)
        res[name] = {"recall_at_L": per_L, "L_for_0.90": L90, "max_hops": hop_limit(hf, L90) if L90 else None,
                     "qps_at_0.90": qps, "fit": rep}
        del ix
    out = {"metric": "recall@10 and QPS at 0.90 on shifted (OOD) queries: LeanVec-OOD (Frank-Wolfe, eigenvector "
                     "search, gradient optimiser) vs LeanVec-ID",
           "workload": f"ood-{n // 1000}k-512, {m} OOD test queries, {m} learning queries, 100k database samples, d=128",
           "results": res, "differentiation": diff, "data": "synthetic"}
    print(json.dumps(out), flush=True)


def ground_truth_big(X, Q, k, qchunk=8192, xchunk=131072):
    """Exact top-k for many queries over a large database (float32, TF32 off), chunked."""
    out = []
    for s in range(0, Q.shape[0], qchunk):
        out.append(ground_truth(X, Q[s:s + qchunk], k, chunk=xchunk))
    return torch.cat(out)


def bench_uneven(args, dev):
    """Uneven batching: 10M x 200 database (text-to-image shape, OOD queries), LeanVec-OOD
    d = 64 LVQ-8; 50k queries with k in {1, 10, 100} and L uniform in [20, 300] (L >= k,
    rerank = L) served by one CUDA-graph launch of the plan the autotuner picks
    (autotune_uneven: the caller's order, longest first, or beam-width classes with their own
    capacities; warps per query, visited-cache slots and warps per block per launch); the
    recall of each beam-width class is reported with its launch."""
    from paper_2312_16335_gb300 import build_lib
    build_lib.build()
    import paper_2312_16335_gb300 as lv
    n, m, D, d = args.n, args.m, 200, 64
    t0 = time.time()
    X, Q, Ql = workloads.make_workload_torch("anisotropic", n, m, D, 1000, cfg=5, device=dev, ood=True,
                                             m_learn=10_000)
    sub = torch.from_numpy(workloads.subsample_rows(n, min(n, 100_000), cfg=5)).to(dev)
    t_data = time.time() - t0
    t0 = time.time()
    A, B, rep = lv.leanvec_fit_ood(X.index_select(0, sub).contiguous(), Ql, d, method=lv.FIT_ES)
    t_fit = time.time() - t0
    t0 = time.time()
    idx = lv.Index(dev.index).encode(X, B, 8, 8, precision=lv.PREC_BF16)
    torch.cuda.synchronize()
    t_enc = time.time() - t0
    t0 = time.time()
    idx.build_graph(R=args.R, L_build=args.L_build, alpha=args.alpha, passes=2, batch=args.batch, rule=args.rule,
                    seed=workloads.SEED_GRAPH + 5)
    clamped = False
    try:
        idx.sync_status()
    except lv.LeanVecError as e:  # a hub target received more reverse edges than the pool holds
        if e.code != -4:
            raise
        clamped = True
    t_build = time.time() - t0
    kl = torch.from_numpy(workloads.uneven_batch(m, seed=workloads.SEED_TEST_QUERIES + 55)).to(dev)
    desc = torch.stack([kl[:, 0], kl[:, 1], kl[:, 1], torch.zeros_like(kl[:, 0])], 1).to(torch.int32).contiguous()
    kmax, Lmax = int(kl[:, 0].max()), int(kl[:, 1].max())
    t0 = time.time()
    truth = ground_truth_big(X, Q, kmax)
    t_truth = time.time() - t0
    log(f"uneven: data {t_data:.1f}s fit {t_fit:.1f}s encode {t_enc:.1f}s build {t_build:.1f}s truth {t_truth:.1f}s")
    # one launch over the whole batch (capacity of the largest L), launch shape tuned
    tune = lv.autotune(idx, Q, A, k=kmax, L=Lmax, rerank=Lmax, desc=desc, width=args.width,
                       projection=lv.PREC_BF16)
    best = tune["best"]
    g1 = lv.SearchGraph(idx, Q, A, k=kmax, L=Lmax, rerank=Lmax, desc=desc, width=args.width,
                        projection=lv.PREC_BF16, hash_slots=best["hash_slots"],
                        warps_per_block=best["warps_per_block"], queries_per_warp=best["queries_per_warp"])
    # the batching form's autotuner: beam-width classes, each with its own capacity, warps per
    # query, visited-cache slots and warps per block, all in one CUDA graph
    plan = lv.autotune_uneven(idx, Q, A, desc, ldo=kmax, width=args.width, projection=lv.PREC_BF16)
    g = lv.UnevenGraph(idx, Q, A, desc, plan, ldo=kmax, width=args.width, projection=lv.PREC_BF16)

    def timed(replay):
        for _ in range(args.warmup):
            replay()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            replay()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.steps

    ms_one = timed(g1.replay)
    with Clocks(dev.index) as clk:
        ms = timed(g.replay)
    ids = g.unsorted(g.ids)
    same = bool((ids == g1.ids).all())  # the tuned classes answer exactly as the one launch
    per = {}
    for kc in sorted(set(kl[:, 0].tolist())):
        sel = kl[:, 0] == kc
        a = ids[sel][:, :kc].long()
        hit = (a.unsqueeze(2) == truth[sel][:, :kc].unsqueeze(1)).any(dim=2) & (a >= 0)
        per[int(kc)] = {"queries": int(sel.sum()), "recall": float(hit.float().mean())}
    for c in plan["plan_launches"]["classes"]:
        sel = plan["plan_orders"]["classes"][c["slice"][0]:c["slice"][1]]
        kk = kl[sel, 0]
        a = ids[sel].long()
        tr = truth[sel]
        hits = 0.0
        for kc in sorted(set(kk.tolist())):
            s2 = kk == kc
            hits += float(((a[s2][:, :kc].unsqueeze(2) == tr[s2][:, :kc].unsqueeze(1)).any(dim=2) &
                           (a[s2][:, :kc] >= 0)).float().sum()) / kc
        c["recall"] = hits / c["queries"]
    tuned_d = uneven_code_width(args, dev, lv, X, Q, Ql, sub, desc, kl, truth, kmax) if args.tune_d else None
    out = {"metric": "QPS of one uneven batch (one CUDA-graph launch) and k-recall@k per class",
           "workload": f"uneven-{n // 1000000}M-200 OOD, {m} queries, k in {{1,10,100}}, L ~ U[20,300], rerank = L",
           "value": m / (ms / 1e3), "unit": "queries/s", "ms_per_batch": ms, "per_k_class": per,
           "tuned_plan": plan["plan"], "plan_ms": plan["plans"], "tuned_launches": plan["classes"],
           "class_launches": plan["plan_launches"]["classes"], "code_width_d": d,
           "code_width_note": "d = 64 is fixed by the configuration; autotune_target_d picks d for an index "
                              "(--workload dsweep)",
           "one_launch": {"qps": m / (ms_one / 1e3), "ms_per_batch": ms_one, "autotune": tune,
                          "same_results_as_classes": same},
           "fit": {k: v for k, v in rep.items() if k != "loss_trace"},
           "setup_seconds": {"data": t_data, "fit": t_fit, "encode": t_enc, "build": t_build, "truth": t_truth},
           "build_reverse_pool_clamped": clamped, "code_width_autotune": tuned_d,
           "clocks": clk.summary(), "data": "synthetic"}
    print(json.dumps(out), flush=True)


def uneven_code_width(args, dev, lv, X, Q, Ql, sub, desc, kl, truth, kmax, ds=(64, 96, 128, 160, 192)):
    """The code width d for the uneven workload by the project's autotuner (autotune_target_d): on
    a graph built once on full-D LVQ-8 codes (so that it does not change with d), for each d the
    LeanVec-OOD eigenvector-search projection is learned, the database encoded, and the smallest L
    with recall@10 >= 0.90 on 10k validation queries (k = 10, max_hops = L) timed; then the uneven
    batch itself on that graph at the configured d and at the tuned d (autotuned plan, per-class
    k-recall@k)."""
    gi = lv.Index(dev.index).set_primary(X, None, 8, X.shape[1])
    t0 = time.time()
    gi.build_graph(R=args.R, L_build=args.L_build, alpha=args.alpha, passes=2, batch=args.batch, rule=args.rule,
                   seed=workloads.SEED_GRAPH + 5)
    try:
        gi.sync_status()
    except lv.LeanVecError as e:
        if e.code != -4:
            raise
    graph, entry = gi.get_graph()
    t_graph = time.time() - t0
    del gi
    Xs = X.index_select(0, sub).contiguous()

    def fit(X_, d_):
        A, B, _ = lv.leanvec_fit_ood(Xs, Ql, d_, method=lv.FIT_ES)
        return A, B

    mv = min(10_000, Q.shape[0])
    tune = lv.autotune_target_d(X, Q[:mv], truth[:mv, :10], graph, entry, ds=ds, k=10, fit=fit, hop_factor=1.0)
    table = [{k_: v for k_, v in r.items() if k_ != "A"} for r in tune["table"]]
    res = {"graph": {"built_on": "full-D LVQ-8 codes", "seconds": t_graph,
                     "mean_degree": float((graph >= 0).sum(1).float().mean())},
           "validation": f"{mv} queries, k = 10, recall@10 >= 0.90, max_hops = L", "table": table,
           "best_d": tune["best"]["d"] if tune["best"] else None, "uneven_batch": {}}
    for d in sorted({64, res["best_d"] or 64}):
        A, B = fit(X, d)
        ix = lv.Index(dev.index).encode(X, B, 8, 8, precision=lv.PREC_BF16).set_graph(graph, entry)
        plan = lv.autotune_uneven(ix, Q, A, desc, ldo=kmax, width=args.width, projection=lv.PREC_BF16)
        g = lv.UnevenGraph(ix, Q, A, desc, plan, ldo=kmax, width=args.width, projection=lv.PREC_BF16)
        for _ in range(3):
            g.replay()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(5):
            g.replay()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 5
        ids = g.unsorted(g.ids)
        per = {}
        for kc in sorted(set(kl[:, 0].tolist())):
            sel = kl[:, 0] == kc
            a = ids[sel][:, :kc].long()
            hit = (a.unsqueeze(2) == truth[sel][:, :kc].unsqueeze(1)).any(dim=2) & (a >= 0)
            per[int(kc)] = float(hit.float().mean())
        res["uneven_batch"][int(d)] = {"qps": Q.shape[0] / (ms / 1e3), "ms": ms, "plan": plan["plan"],
                                       "k_recall_at_k": per}
        del g, ix
    return res


def bench_precision(args, dev):
    """Precision form at 10M: 10M x 768 (10,000 components), d = 160 LVQ-4 primaries + LVQ-8
    secondaries, R = 64; second moments in bf16 (tcgen05) with FP64 eig; query and database
    projection in e4m3 with per-row scales (tcgen05 f8f6f4); 100k queries.  Errors of the
    reduced-precision steps are stated against FP64 references on samples."""
    from paper_2312_16335_gb300 import build_lib
    build_lib.build()
    import paper_2312_16335_gb300 as lv
    n, m, D, d = args.n, args.m, 768, 160
    t0 = time.time()
    X, Q, _ = workloads.make_workload_torch("anisotropic", n, m, D, 10_000, cfg=4, device=dev, m_learn=0)
    t_data = time.time() - t0
    sub = torch.from_numpy(workloads.subsample_rows(n, 100_000, cfg=4)).to(dev)
    Xs = X.index_select(0, sub).contiguous()
    # second moments: bf16 tensor cores vs FP64 (NumPy) on the 100k sample
    K16 = lv.leanvec_second_moment(Xs, precision=lv.PREC_BF16).double().cpu().numpy()
    Xs64 = Xs.double().cpu().numpy()
    K64 = Xs64.T @ Xs64
    nrm = np.linalg.norm(Xs64, axis=0)
    k_err = float(np.abs(K16 - K64).max() / np.outer(nrm, nrm).max())
    t0 = time.time()
    A = lv.leanvec_fit_id(Xs, d, precision=lv.PREC_BF16)
    t_fit = time.time() - t0
    A32 = lv.leanvec_fit_id(Xs, d, precision=lv.PREC_FP32)
    A64 = np.linalg.eigh(K64)[1][:, ::-1][:, :d].T
    proj = lambda P: P.T @ P
    sub_err = float(np.linalg.norm(proj(A.double().cpu().numpy()) - proj(A64)) / np.sqrt(d))
    # projection: e4m3 vs FP64 on 2000 queries, relative to ||q|| ||a||
    qs = Q[:2000].contiguous()
    Y8 = lv.leanvec_project(qs, A, precision=lv.PREC_FP8).double().cpu().numpy()
    Yr = qs.double().cpu().numpy() @ A.double().cpu().numpy().T
    sc = np.linalg.norm(qs.double().cpu().numpy(), axis=1)[:, None] * np.linalg.norm(A.double().cpu().numpy(), axis=1)[None, :]
    p_err = {"max": float((np.abs(Y8 - Yr) / sc).max()), "mean": float((np.abs(Y8 - Yr) / sc).mean())}
    del K16, Xs64, Y8, Yr
    t0 = time.time()
    idx = lv.Index(dev.index).encode(X, A, primary_bits=4, secondary_bits=8, precision=lv.PREC_FP8)
    torch.cuda.synchronize()
    t_enc = time.time() - t0
    t0 = time.time()
    # the searched graph: built on LVQ-8 codes of the unreduced vectors (the full-precision
    # stand-in, as the id workload's), or with --graph primary on the LVQ-4 primaries
    gi = lv.Index(dev.index).set_primary(X, None, 8, D) if args.graph == "full" else idx
    gi.build_graph(R=args.R, L_build=args.L_build, alpha=args.alpha, passes=2, batch=args.batch, rule=args.rule,
                   seed=workloads.SEED_GRAPH + 4)
    clamped = False
    try:
        gi.sync_status()
    except lv.LeanVecError as e:
        if e.code != -4:
            raise
        clamped = True
    if gi is not idx:
        idx.set_graph(*gi.get_graph())
        del gi
    torch.cuda.synchronize()
    t_build = time.time() - t0
    mt = min(10_000, m)
    truth = ground_truth_big(X, Q[:mt], 10)
    res = {}
    for pname, prec in (("fp8", lv.PREC_FP8), ("fp32", lv.PREC_FP32)):
        L90, trace = calibrate(lambda L: idx.search(Q[:mt], A, k=10, L=L, rerank=L, width=args.width,
                                                     projection=prec)[0], truth, 10)
        L90 = L90 or L_GRID[-1]
        nst = max(3, args.steps // 5)
        ms, _ = time_steps(lambda ev: idx.search(Q, A, k=10, L=L90, rerank=L90, width=args.width, projection=prec),
                           nst, 2)
        res[pname] = {"L_for_0.90": L90, "recall_trace": trace, "qps": m * nst / (ms / 1e3)}
    diag = precision_diagnosis(args, dev, lv, X, Q, A, idx, truth[:1000]) if args.diagnose else None
    out = {"metric": "QPS at 10-recall@10 = 0.90 with FP8 (e4m3, per-row scaled) query projection; "
                     "precision errors vs FP64",
           "workload": f"prec-{n // 1000000}M-768: 10,000-component mixture, {m} queries (recall on {mt}), "
                       f"d=160 LVQ-4 primary + LVQ-8 secondary, R={args.R}, L_build={args.L_build}, "
                       f"alpha={args.alpha} (rule {args.rule}), graph built on "
                       f"{'full-D LVQ-8 codes' if args.graph == 'full' else 'the LVQ-4 primaries'}",
           "results": res,
           "errors_vs_fp64": {"second_moment_bf16_max_rel": k_err, "fit_id_bf16_projector_dist": sub_err,
                              "projection_fp8_rel_to_norms": p_err},
           "setup_seconds": {"data": t_data, "fit": t_fit, "encode_fp8": t_enc, "build": t_build},
           "build_reverse_pool_clamped": clamped, "diagnosis": diag, "data": "synthetic"}
    print(json.dumps(out), flush=True)


def precision_diagnosis(args, dev, lv, X, Q, A, idx, truth, rs=(64, 128, 256, 512)):
    """Where prec-10M-768's recall is lost, on the first 1000 queries: the fraction of the true top
    10 that the top r of an exhaustive ranking by primary score contains -- with float32 projected
    vectors (the d = 160 projection's ceiling) and with the decoded LVQ-4 primaries of the index (the
    quantisation's) -- and the search on the searched graph and on the other one (built on the LVQ-4
    primaries or on full-D LVQ-8 codes): the graph's share."""
    mq = truth.shape[0]
    qp = Q[:mq] @ A.T
    # decoded LVQ-4 primaries: code 2j in the low nibble, 2j + 1 in the high one; constants
    # {delta, lower} right after the code chunks
    inf = idx.info()
    d = inf["d"]
    rec = idx.primary_records()
    cb = -(-((d + 1) // 2) // 16) * 16
    mean = idx.primary_mean()
    best = {"float32": None, "lvq4": None}
    for name in best:
        vals, ids = [], []
        for s0 in range(0, X.shape[0], 1 << 20):
            if name == "float32":
                Y = X[s0:s0 + (1 << 20)] @ A.T
            else:
                r = rec[s0:s0 + (1 << 20)]
                codes = torch.stack([r[:, :cb] & 15, r[:, :cb] >> 4], dim=2).reshape(r.shape[0], 2 * cb)[:, :d].float()
                c = r[:, cb:cb + 8].contiguous().view(torch.float32)
                Y = mean[None, :] + c[:, 1:2] + c[:, 0:1] * codes
            S = qp @ Y.T
            v, i = torch.topk(S, max(rs), dim=1)
            vals.append(v)
            ids.append(i + s0)
        v, i = torch.topk(torch.cat(vals, 1), max(rs), dim=1)
        best[name] = torch.gather(torch.cat(ids, 1), 1, i)
    ceiling = {name: {r: float((b[:, :r].unsqueeze(2) == truth[:, :10].unsqueeze(1)).any(dim=1).float().mean())
                      for r in rs} for name, b in best.items()}
    # the same search on the other graph: built on the LVQ-4 primaries when the searched one is on
    # full-D LVQ-8 codes, and the other way round (alpha, rule, R, L_build as configured)
    other = "primary" if args.graph == "full" else "full"
    gi = lv.Index(dev.index).set_primary(X, None, 8, X.shape[1]) if other == "full" else lv.Index(dev.index)
    if other == "primary":
        gi.encode(X, A, primary_bits=4, secondary_bits=0, precision=lv.PREC_FP8)
    t0 = time.time()
    gi.build_graph(R=args.R, L_build=args.L_build, alpha=args.alpha, passes=2, batch=args.batch, rule=args.rule,
                   seed=workloads.SEED_GRAPH + 4)
    try:
        gi.sync_status()
    except lv.LeanVecError as e:
        if e.code != -4:
            raise
    g, e = gi.get_graph()
    t_other = time.time() - t0
    del gi
    g0, e0 = idx.get_graph()

    def trace_of():
        out = []
        for L in (128, 256, 384, 512):
            ids = idx.search(Q[:mq], A, k=10, L=L, rerank=L, width=args.width, projection=lv.PREC_FP8)[0]
            out.append((L, recall_at(ids, truth, 10)))
        return out

    searched = {"graph": args.graph, "mean_degree": float((g0 >= 0).sum(1).float().mean()),
                "recall_trace_fp8": trace_of()}
    idx.set_graph(g, e)
    alt = {"graph": other, "build_seconds": t_other, "mean_degree": float((g >= 0).sum(1).float().mean()),
           "recall_trace_fp8": trace_of()}
    idx.set_graph(g0, e0)
    return {"queries": mq, "exhaustive_primary_ceiling": ceiling, "searched_graph": searched, "other_graph": alt}


def bench_buildstudy(args, dev):
    """Graph construction on primaries vs on (near) full precision: the graph is built once on the
    d = 160 LVQ-8 primaries and once on LVQ-8 codes of the unreduced D-dimensional vectors (0.4 %
    quantisation error: the full-precision stand-in), same R, L_build, alpha, passes, batch and
    seed; then both the LeanVec search and the full-D FP32 search are calibrated for recall 0.90 on
    each graph."""
    args.graph = "primary"  # setup builds the primary graph; the full-D one is built below
    S = setup(args, dev)
    lv, X, Q, A, truth = S["lv"], S["X"], S["Q"], S["A"], S["truth"]
    idx, base = S["idx"], S["base"]
    proj = lv.PREC_BF16 if args.projection == "bf16" else lv.PREC_FP32
    t0 = time.time()
    full = lv.Index(dev.index).set_primary(X, None, 8, args.D)
    torch.cuda.synchronize()
    t_enc_full = time.time() - t0
    t0 = time.time()
    full.build_graph(R=args.R, L_build=args.L_build, alpha=args.alpha, passes=2, batch=args.batch, rule=args.rule,
                     seed=workloads.SEED_GRAPH + 2)
    clamped = False
    try:
        full.sync_status()
    except lv.LeanVecError as e:  # reverse-edge pool clamp: the build completed, some reverse edges dropped
        if e.code != -4:
            raise
        clamped = True
    t_build_full = time.time() - t0
    graphs = {"primary_d%d" % args.d: (S["graph"], S["entry"]), "full_D_lvq8": full.get_graph()}
    del full
    res = {}
    for name, (g, e) in graphs.items():
        r = {"mean_degree": float((g >= 0).sum(1).float().mean())}
        for arm, ix, fn in (("leanvec", idx, lambda L: idx.search(Q, A, k=10, L=L, rerank=L, width=args.width,
                                                                   projection=proj)),
                            ("fp32", base, lambda L: base.search(Q, None, k=10, L=L, width=args.width))):
            ix.set_graph(g, e)
            L, trace = calibrate(lambda L: fn(L)[0], truth, 10)
            a = {"L_for_0.90": L, "recall_trace": trace[-3:]}
            if L:
                nst = max(5, args.steps // 5)
                ms, _ = time_steps(lambda ev: fn(L), nst, 2)
                a["qps"] = args.m * nst / (ms / 1e3)
            r[arm] = a
        res[name] = r
        log(f"{name}: {r}")
    out = {"metric": "graph construction on d = %d primaries vs on full-D LVQ-8 codes: build seconds, and QPS "
                     "at recall@10 = 0.90 of the LeanVec and full-D FP32 searches on each graph" % args.d,
           "workload": f"id-{args.n // 1000}k-{args.D}, {args.m} ID queries, R={args.R}, L_build={args.L_build}, "
                       f"alpha={args.alpha}, prune rule {args.rule}, 2 passes, batch {args.batch}",
           "build_seconds": {"primary_d%d" % args.d: S["t_build"], "full_D_lvq8": t_build_full},
           "encode_seconds": {"primary_d%d" % args.d: S["t_enc"] + S["t_fit"], "full_D_lvq8": t_enc_full},
           "full_D_reverse_pool_clamped": clamped, "results": res, "data": "synthetic"}
    print(json.dumps(out), flush=True)


def bench_l2(args, dev):
    """Euclidean workload shaped like gist-960-1M (Table 1: D = 960, Euclidean, d = 160): the
    anisotropic mixture without normalisation (norms vary with the component), 10k ID queries,
    ground truth = the 10 nearest in L2.  One graph, built in an L2 index on full-D LVQ-8 codes with
    Vamana's rule on squared distances (alpha-scaled, alpha = 1.2 as the paper sets for L2); then
    the LeanVec search (LVQ-8 primaries of d dims + LVQ-8 secondaries, scores 2 <Aq, y> - ||x||^2,
    rerank 2 <q, x> - ||x||^2) and the full-D FP32 search, each at the smallest grid L with
    recall@10 >= 0.90."""
    from paper_2312_16335_gb300 import build_lib
    build_lib.build()
    import paper_2312_16335_gb300 as lv
    t0 = time.time()
    X, Q, _ = workloads.make_workload_torch("anisotropic", args.n, args.m, args.D, args.components, cfg=4,
                                            device=dev, normalize=False)
    torch.cuda.synchronize()
    nrm = X.norm(dim=1)
    log(f"data {tuple(X.shape)} queries {tuple(Q.shape)} in {time.time() - t0:.1f}s; ||x|| mean "
        f"{float(nrm.mean()):.2f} sd {float(nrm.std()):.2f}")
    t0 = time.time()
    sub = torch.from_numpy(workloads.subsample_rows(args.n, min(args.n, 100_000), cfg=4)).to(dev)
    A = lv.leanvec_fit_id(X.index_select(0, sub).contiguous(), args.d)
    idx = lv.Index(dev.index, metric=lv.METRIC_L2).encode(
        X, A, primary_bits=8, secondary_bits=16 if args.secondary == "fp16" else 8)
    torch.cuda.synchronize()
    t_enc = time.time() - t0
    t0 = time.time()
    gi = lv.Index(dev.index, metric=lv.METRIC_L2)
    if args.graph == "full":
        gi.set_primary(X, None, 8, args.D)
    else:
        gi = idx
    gi.build_graph(R=args.R, L_build=args.L_build, alpha=args.alpha, passes=2, batch=args.batch, rule=args.rule,
                   seed=workloads.SEED_GRAPH + 4)
    clamped = False
    try:
        gi.sync_status()
    except lv.LeanVecError as e:  # reverse-edge pool clamp: the build completed, some reverse edges dropped
        if e.code != -4:
            raise
        clamped = True
    graph, entry = gi.get_graph()
    if gi is not idx:
        idx.set_graph(graph, entry)
        del gi
    torch.cuda.synchronize()
    t_build = time.time() - t0
    log(f"fit+encode {t_enc:.2f}s build {t_build:.2f}s")
    base = lv.Index(dev.index, metric=lv.METRIC_L2).encode_fp32(X).set_graph(graph, entry)
    truth = ground_truth(X, Q, 10, l2=True)
    truth_ip = ground_truth(X, Q, 10)
    proj = lv.PREC_BF16 if args.projection == "bf16" else lv.PREC_FP32
    res = {"mean_degree": float((graph >= 0).sum(1).float().mean()),
           "ip_top10_overlap": recall_at(truth_ip, truth, 10)}
    hf = args.hop_factor
    for arm, fn in (("leanvec", lambda L: idx.search(Q, A, k=10, L=L, rerank=L, max_hops=hop_limit(hf, L),
                                                     width=args.width, projection=proj)),
                    ("fp32", lambda L: base.search(Q, None, k=10, L=L, max_hops=hop_limit(hf, L), width=args.width))):
        L, trace = calibrate(lambda L: fn(L)[0], truth, 10)
        a = {"L_for_0.90": L, "max_hops": hop_limit(hf, L) if L else None, "recall_trace": trace[-3:]}
        if L:
            nst = max(5, args.steps // 5)
            ms, _ = time_steps(lambda ev: fn(L), nst, 3)
            a["qps"] = args.m * nst / (ms / 1e3)
        res[arm] = a
        log(f"{arm}: {a}")
    out = {"metric": "QPS at 10-recall@10 = 0.90 under the Euclidean distance, LeanVec vs full-D FP32 graph search",
           "workload": f"l2-{args.n // 1000}k-{args.D} (gist-960-1M shape): anisotropic Gaussian mixture "
                       f"({args.components} components, i^-1 spectrum), not normalised; {args.m} ID queries; "
                       f"LeanVec-ID d={args.d}, LVQ-8 primary + {'FP16' if args.secondary == 'fp16' else 'LVQ-8'} secondary; graph R={args.R}, "
                       f"L_build={args.L_build}, alpha={args.alpha} (rule {args.rule}), batch {args.batch}, built in an L2 index on "
                       f"{'full-D LVQ-8 codes' if args.graph == 'full' else 'the primaries'}; k=10, rerank=L, "
                       f"max_hops=ceil({args.hop_factor} L) (both arms)",
           "build_seconds": t_build, "encode_seconds": t_enc, "reverse_pool_clamped": clamped, "results": res,
           "data": "synthetic"}
    print(json.dumps(out), flush=True)


def l2_bandwidth(dev, mb=32, reps=200):
    """Measured L2 bandwidth: a device copy between two L2-resident buffers (2 x mb MB, far below
    the L2 size), replayed `reps` times from one CUDA graph so that launch gaps do not count;
    bytes read + written per second (the best of three replays)."""
    n = mb * (1 << 20) // 4
    a = torch.ones(n, device=dev)
    b = torch.empty_like(a)
    s = torch.cuda.Stream(device=dev)
    s.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(s):
        for _ in range(3):
            b.copy_(a)
    torch.cuda.current_stream(dev).wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        for _ in range(reps):
            b.copy_(a)
    best = None
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        g.replay()
        e1.record()
        torch.cuda.synchronize()
        gbs = 2 * 4 * n * reps / (e0.elapsed_time(e1) / 1e3) / 1e9
        best = gbs if best is None else max(best, gbs)
    return best


def bench_c1(args, dev):
    """id-10k-128, the L2-resident configuration: 10k x 128 isotropic mixture (100 components,
    sigma 0.3, unit norm), 1000 ID queries, LeanVec-ID d = 32 (PCA of the full database), LVQ-8
    primary + LVQ-8 secondary, GPU-built graph R = 32, L_build = 64, alpha = 0.95 (alpha-scaled
    rule), k = 10, L = rerank = 50.  The index (about 3 MB) stays in L2, so the roofline is the
    L2 bandwidth measured in this run, and L2 is flushed (a 256 MB write) before every timed step.
    Also reported: the same search on the graph built with the benchmark's default rule (unit-norm
    L2 rule, alpha 1.02), at L = 50 and at the smallest L with recall@10 >= 0.90, and a batch of
    100k queries from the same mixture (the configured 1000 fill a fraction of one wave)."""
    from paper_2312_16335_gb300 import build_lib
    build_lib.build()
    import paper_2312_16335_gb300 as lv
    import oracle
    from oracle import rounding
    n, D, d, k = 10_000, 128, 32, 10
    big = 100_000
    w = workloads.make_workload("isotropic", n, big, D, 100, cfg=1, sigma=0.3, m_learn=0)
    X = torch.from_numpy(w.X).to(dev)
    Qall = torch.from_numpy(w.Q).to(dev)
    A = lv.leanvec_fit_id(X, d)
    proj = lv.PREC_BF16 if args.projection == "bf16" else lv.PREC_FP32
    flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)  # 256 MB > L2
    truth_all = ground_truth(X, Qall, k)
    l2_gbs = l2_bandwidth(dev)
    Ah = A.cpu().numpy()
    Y = (w.X.astype(np.float64) @ Ah.astype(np.float64).T).astype(np.float32)
    prim = oracle.lvq_encode(Y, oracle.mean_fp32(Y), 8)
    sec = oracle.lvq_encode(w.X, oracle.mean_fp32(w.X), 8)
    st_ = torch.cuda.current_stream(dev)

    def timed(idx, Q, L):
        m = Q.shape[0]
        ids_buf = torch.empty((m, k), dtype=torch.int32, device=dev)
        sc_buf = torch.empty((m, k), dtype=torch.float32, device=dev)

        def search(ev=None, stats=False):
            return idx.search(Q, A, k=k, L=L, rerank=L, width=args.width, projection=proj, out=(ids_buf, sc_buf),
                              events=ev, stats=stats, queries_per_warp=args.qpw, visited_bits=args.vbits)
        for _ in range(5):
            search()
        times, kern = [], []
        for _ in range(args.steps):
            flush.fill_(1.0)
            ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            ev[0].record(st_)
            ev[1].record(st_)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st_)
            search(ev)
            e1.record(st_)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
            kern.append(ev[0].elapsed_time(ev[1]))
        _, _, st = search(stats=True)
        return ids_buf, statistics.median(times), statistics.median(kern), float(st[:, 1].double().mean())

    def run(rule, alpha, L_fixed, m):
        idx = lv.Index(dev.index).encode(X, A, primary_bits=8, secondary_bits=8)
        idx.build_graph(R=32, L_build=64, alpha=alpha, passes=2, batch=1024, rule=rule, seed=workloads.SEED_GRAPH + 1)
        idx.sync_status()
        graph, entry = idx.get_graph()
        Q, truth = Qall[:m], truth_all[:m]
        if L_fixed:
            L = L_fixed
        else:
            L, _ = calibrate(lambda L: idx.search(Q, A, k=k, L=L, rerank=L, width=args.width, projection=proj)[0],
                             truth, k)
            L = L or L_GRID[-1]
        ids, step_ms, kern_ms, scored_gpu = timed(idx, Q, L)
        rec = recall_at(ids, truth, k)
        # the method's own bytes and the parity of ids: the oracle on (up to) the first 1000 queries
        mo = min(m, 1000)
        t0 = time.perf_counter()
        r = oracle.search(graph.cpu().numpy(), entry, rounding.project(w.Q[:mo], Ah, args.projection), k=k, L=L,
                          rerank=L, prim=prim, sec=sec, qs=w.Q[:mo].astype(np.float64), width=args.width)
        cpu_s = time.perf_counter() - t0
        bq = method_bytes_per_query(D, d, 8, 32, float(r["hops"].mean()), float(r["scored"].mean()), L)
        achieved = bq * m / (kern_ms / 1e3) / 1e9
        return idx, {"graph": f"rule {rule}, alpha {alpha}", "mean_degree": float((graph >= 0).sum(1).float().mean()),
                     "queries": m, "L": L, "recall_at_10": rec, "qps": m / (step_ms / 1e3), "step_ms": step_ms,
                     "ids_equal_oracle": float((ids[:mo].cpu().numpy() == r["ids"]).mean()),
                     "roofline": {"bound": "l2", "achieved": achieved, "peak": l2_gbs, "unit": "GB/s",
                                  "frac": achieved / l2_gbs, "kernel_ms": kern_ms, "bytes_per_query": bq,
                                  "hops_per_query": float(r["hops"].mean()),
                                  "scored_per_query": float(r["scored"].mean()), "gpu_scored_per_query": scored_gpu},
                     "cpu_oracle_qps": mo / cpu_s}

    idx, main = run(0, 0.95, 50, 1000)
    others = [run(0, 0.95, 50, big)[1], run(1, 1.02, 50, 1000)[1], run(1, 1.02, 0, 1000)[1],
              run(1, 1.02, 0, big)[1]]
    # e2e through the C ABI with host buffers (one call per step) on the configured case
    Qh = Qall[:1000].cpu().pin_memory()
    ids_h = torch.empty((1000, k), dtype=torch.int32).pin_memory()
    sc_h = torch.empty((1000, k), dtype=torch.float32).pin_memory()
    for _ in range(3):
        idx.search_host(Qh, A, k=k, L=50, rerank=50, width=args.width, projection=proj, out=(ids_h, sc_h))
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        idx.search_host(Qh, A, k=k, L=50, rerank=50, width=args.width, projection=proj, out=(ids_h, sc_h))
    e1.record()
    torch.cuda.synchronize()
    e2e = 1000 * args.steps / (e0.elapsed_time(e1) / 1e3)
    out = {"metric": "QPS at k=10, L = rerank = 50 (recall@10 reported), id-10k-128; L2 GB/s",
           "value": main["qps"], "unit": "queries/s", "n_gpus": 1, "steps": args.steps,
           "higher_is_better": True, "dtype": "f32 (u8 LVQ codes decoded to f32)", "data": "synthetic",
           "config": {"workload": "id-10k-128: isotropic Gaussian mixture (100 components, sigma 0.3), unit norm, "
                                  "inner product; 1000 ID queries; LeanVec-ID d=32, LVQ-8 primary + LVQ-8 "
                                  "secondary; GPU-built graph R=32, L_build=64, alpha=0.95 (alpha-scaled rule); "
                                  "k=10, L=rerank=50, no expansion budget",
                      "projection": args.projection, "width": args.width, "queries_per_warp": args.qpw or 1, "visited_bits": args.vbits or "default",
                      "l2": "index about 3 MB, L2-resident; L2 flushed (256 MB written) before every timed step"},
           "recall_at_10": main["recall_at_10"], "ids_equal_oracle": main["ids_equal_oracle"],
           "e2e": {"value": e2e, "unit": "queries/s", "h2d_bytes_per_step": 1000 * D * 4,
                   "d2h_bytes_per_step": 1000 * k * 8, "api": "leanvec_search_host (C ABI), one call per step"},
           "roofline": dict(main["roofline"], kernel="beam_kernel + rerank_kernel",
                            peak_kind="measured in this run: L2-resident device copy (2 x 32 MB, graph-replayed)",
                            note="1000 queries fill a fraction of one wave of the persistent grid's query slots (one "
                                 "warp each): the step is the latency of the longest searches; see the 100k-query rows"),
           "cpu_baseline": {"value": main["cpu_oracle_qps"], "unit": "queries/s", "cores": os.cpu_count(),
                            "kind": "oracle", "sample": "all 1000 queries"},
           "other_rows": others}
    print(json.dumps(out), flush=True)


def bench_loss(args, dev):
    """The differentiation form alone (Sec. 2.2 problem "leanvec_orthonormal", Eq. "leanvec_gradients"
    per pair): the pair loss forward and backward over --m learning queries x --n database samples
    (default 10^4 x 10^5, 10^9 pairs), D = 512, d = 128, `steps` of each after `warmup`, timed with
    CUDA events; the timed calls sit inside an NVTX range 'timed' for launch lists."""
    from paper_2312_16335_gb300 import build_lib
    build_lib.build()
    import paper_2312_16335_gb300 as lv
    pk = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    bf16 = float(pk.get("bf16_tflops", 1900.0))
    src = "measured" if "bf16_tflops" in pk else "fallback"
    tf32_peak = bf16 * 1.1 / 2.25
    Xo, _, Qo = workloads.make_workload_torch("anisotropic", args.n, 1000, 512, args.components, cfg=3, device=dev,
                                              ood=True, m_learn=args.m)
    Ai = lv.leanvec_fit_id(Xo, 128)
    m, n, D, d = Qo.shape[0], Xo.shape[0], 512, 128
    for _ in range(max(1, args.warmup)):
        lv.leanvec_ood_loss_fwd(Ai, Ai, Qo, Xo)
        lv.leanvec_ood_loss_bwd(Ai, Ai, Qo, Xo)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    tf = tb = 0.0
    for _ in range(args.steps):
        torch.cuda.nvtx.range_push("timed")
        ev[0].record()
        L = lv.leanvec_ood_loss_fwd(Ai, Ai, Qo, Xo)
        ev[1].record()
        lv.leanvec_ood_loss_bwd(Ai, Ai, Qo, Xo)
        ev[2].record()
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        tf += ev[0].elapsed_time(ev[1]) / 1e3
        tb += ev[1].elapsed_time(ev[2]) / 1e3
    tf /= args.steps
    tb /= args.steps
    # forward: tf32x3 tile products (three tf32 MMAs per product over K = D)
    ex_f = 3 * 2.0 * m * n * D
    # backward: two passes (U = R X', V = R^T Q'), each recomputing R in bf16x3 (three bf16 MMAs
    # over K = D) and contracting it in tf32x3 (three tf32 MMAs over the d outputs); then the
    # tf32x3 gradient GEMMs U^T Q, V^T X
    bf_b = 2 * 3 * 2.0 * m * n * D
    tf_b = 2 * 3 * 2.0 * m * n * d + 3 * 2.0 * D * d * (m + n)
    ideal_b = bf_b / (bf16 * 1e12) + tf_b / (tf32_peak * 1e12)
    out = {"metric": "pair loss forward / backward, seconds per call (tensor cores)", "data": "synthetic",
           "workload": f"ood-{n // 1000}k-512: {m} learning queries x {n} database samples, d = 128, "
                       "A = B = LeanVec-ID",
           "steps": args.steps, "warmup": args.warmup, "loss": L,
           "forward": {"seconds": tf, "executed_tflops": ex_f / tf / 1e12, "frac": ex_f / tf / 1e12 / tf32_peak,
                       "bound": "tensor (tf32, three MMAs per product)"},
           "backward": {"seconds": tb, "executed_bf16_tflop": bf_b / 1e12, "executed_tf32_tflop": tf_b / 1e12,
                        "ideal_seconds": ideal_b, "frac": ideal_b / tb,
                        "bound": "tensor (bf16x3 residual tiles + tf32x3 contractions; frac = time at the "
                                 "peaks / measured time)"},
           "peak_tflops": {"bf16": bf16, "tf32": tf32_peak},
           "peak_source": src + " bf16; tf32 = measured bf16 x nominal tf32/bf16 ratio"}
    print(json.dumps(out), flush=True)


def bench_kernels(args, dev):
    """The offline and auxiliary kernels of the path, each timed alone through its C-ABI call
    (CUDA events on the launching stream, warm-up first) and set against its roofline:
    second moments and projections (tcgen05 GEMMs), LVQ encode and column mean (HBM), FP64
    Jacobi eigh, LeanVec-ID / -OOD fits, the pair loss forward + backward (tf32x3 tensor cores)."""
    from paper_2312_16335_gb300 import build_lib
    build_lib.build()
    import paper_2312_16335_gb300 as lv
    hbm, hbm_src = peaks()
    pk = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    bf16 = float(pk.get("bf16_tflops", 1900.0))
    src = "measured" if "bf16_tflops" in pk else "fallback"
    # CUDA-core FP32 peak: 152 SMs x 128 lanes x 2 flops x 2.07 GHz (nominal; nothing measures it here)
    fp32_cc = 152 * 128 * 2 * 2.07e9 / 1e12

    def timed(fn, reps):
        fn()
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps / 1e3  # seconds per call

    res = {}

    def tensor_row(name, flops, t, peak, unit_peak_src):
        res[name] = {"seconds": t, "bound": "tensor", "achieved_tflops": flops / t / 1e12, "peak_tflops": peak,
                     "frac": flops / t / 1e12 / peak, "peak_source": unit_peak_src}
        log(name, res[name])

    def hbm_row(name, nbytes, t):
        res[name] = {"seconds": t, "bound": "hbm", "achieved_gbs": nbytes / t / 1e9, "peak_gbs": hbm,
                     "frac": nbytes / t / 1e9 / hbm, "algorithmic_bytes": nbytes, "peak_source": hbm_src}
        log(name, res[name])

    n, D, d = args.n, args.D, args.d
    X, Q, Ql = workloads.make_workload_torch("anisotropic", n, args.m, D, args.components, cfg=2, device=dev)
    torch.cuda.synchronize()
    # a13: second moments K = sum x x^T (bf16 operands, tcgen05, FP32 accumulation); K is symmetric,
    # so the algorithmic flops are 2 n per distinct entry: n D (D + 1)
    for ns in (100_000, n):
        Xs = X[:ns]
        t = timed(lambda: lv.leanvec_second_moment(Xs, precision=lv.PREC_BF16), 5)
        tensor_row(f"second_moment_bf16_{ns // 1000}k_x_{D}", float(ns) * D * (D + 1), t, bf16, src)
        res[f"second_moment_bf16_{ns // 1000}k_x_{D}"]["hbm_frac"] = 4.0 * ns * D / t / 1e9 / hbm
        res[f"second_moment_bf16_{ns // 1000}k_x_{D}"]["tflops_as_full_product"] = 2.0 * ns * D * D / t / 1e12
    t = timed(lambda: lv.leanvec_second_moment(X[:100_000], precision=lv.PREC_FP32), 3)
    res[f"second_moment_fp32_100k_x_{D}"] = {"seconds": t, "tflops": 2.0 * 100_000 * D * D / t / 1e12,
                                             "bound": "fp32 CUDA cores", "peak_tflops_nominal": fp32_cc}
    log("second_moment_fp32", res[f"second_moment_fp32_100k_x_{D}"])
    # a1 / a11: projections x -> B x of the database (and q -> A q of a search batch)
    A = lv.leanvec_fit_id(X[:100_000], d)
    ldy = (d + 15) // 16 * 16
    for prec, tag in ((lv.PREC_BF16, "bf16"), (lv.PREC_FP8, "fp8"), (lv.PREC_TF32X3, "tf32x3"), (lv.PREC_FP32, "fp32")):
        t = timed(lambda: lv.leanvec_project(X, A, ldy=ldy, precision=prec), 5)
        # algorithmic bytes: read X (float32), write Y (float32); the GEMM itself is 2 n D d flops
        hbm_row(f"project_{tag}_{n // 1000}k_{D}_to_{d}", 4.0 * n * D + 4.0 * n * ldy, t)
        res[f"project_{tag}_{n // 1000}k_{D}_to_{d}"]["tflops"] = 2.0 * n * D * d / t / 1e12
    for prec, tag in ((lv.PREC_BF16, "bf16"), (lv.PREC_FP8, "fp8")):
        t = timed(lambda: lv.leanvec_project(Q, A, ldy=ldy, precision=prec), 20)
        hbm_row(f"project_{tag}_queries_{Q.shape[0] // 1000}k_{D}_to_{d}", 4.0 * Q.shape[0] * (D + ldy), t)
    # a11: column mean and LVQ-8 encode of the full-D vectors (secondaries)
    mu = lv.leanvec_column_mean(X)
    t = timed(lambda: lv.leanvec_column_mean(X), 5)
    hbm_row(f"column_mean_{n // 1000}k_{D}", 4.0 * n * D, t)
    stride = lv.leanvec_record_stride(D, 8)
    t = timed(lambda: lv.leanvec_lvq_encode(X, mu, 8), 5)
    hbm_row(f"lvq8_encode_{n // 1000}k_{D}", 4.0 * n * D + float(n) * stride, t)
    Y = lv.leanvec_project(X, A, ldy=d, precision=lv.PREC_FP32)
    muy = lv.leanvec_column_mean(Y)
    t = timed(lambda: lv.leanvec_lvq_encode(Y, muy, 8), 5)
    hbm_row(f"lvq8_encode_{n // 1000}k_{d}", 4.0 * n * d + float(n) * lv.leanvec_record_stride(d, 8), t)
    del Y
    # a14: FP64 Jacobi eigh of a D x D second moment; LeanVec-ID fit end to end
    K = lv.leanvec_second_moment(X[:100_000], precision=lv.PREC_FP32).double()
    t = timed(lambda: lv.leanvec_eigh(K), 1)
    res[f"eigh_fp64_{D}"] = {"seconds": t, "method": "cyclic Jacobi, all D pairs"}
    log("eigh", res[f"eigh_fp64_{D}"])
    t = timed(lambda: lv.leanvec_eigh_top(K, d), 3)
    res[f"eigh_top_fp64_{D}_{d}"] = {"seconds": t, "method": "tridiagonal reduction + bisection + inverse "
                                     "iteration, the d leading pairs (the fits' path)"}
    log("eigh_top", res[f"eigh_top_fp64_{D}_{d}"])
    t = timed(lambda: lv.leanvec_fit_id(X[:100_000], d, precision=lv.PREC_BF16), 1)
    res[f"fit_id_bf16_100k_{D}_to_{d}"] = {"seconds": t}
    log("fit_id", res[f"fit_id_bf16_100k_{D}_to_{d}"])
    # a14 / a15 on the OOD shape: 100k database samples, 10k learning queries, D = 512, d = 128
    Xo, _, Qo = workloads.make_workload_torch("anisotropic", 100_000, 1000, 512, args.components, cfg=3, device=dev,
                                              ood=True, m_learn=10_000)
    for meth, tag in ((lv.FIT_FW, "fw"), (lv.FIT_ES, "es")):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, _, rep = lv.leanvec_fit_ood(Xo, Qo, 128, method=meth)
        torch.cuda.synchronize()
        res[f"fit_ood_{tag}_100k_10k_512_to_128"] = {"seconds": time.perf_counter() - t0,
                                                      "iterations": rep["iterations"]}
        log(tag, res[f"fit_ood_{tag}_100k_10k_512_to_128"])
    Ai = lv.leanvec_fit_id(Xo, 128)
    pair_flops = 2.0 * Qo.shape[0] * Xo.shape[0] * (512 + 128)  # q^T x and (A q)^T (B x) per pair
    t = timed(lambda: lv.leanvec_ood_loss_fwd(Ai, Ai, Qo, Xo), 2)
    # the forward runs r = qt^T x (qt = q - B^T A q) as three tf32 tensor-core products per pair
    # (hi/lo splits): 3 x 2 m n D executed flops against the tf32 peak (bf16 measured x 1.1 / 2.25)
    tf32_peak = bf16 * 1.1 / 2.25
    exec_flops = 3 * 2.0 * Qo.shape[0] * Xo.shape[0] * 512
    res["pair_loss_fwd_10k_x_100k_512_128"] = {"seconds": t, "pair_tflops": pair_flops / t / 1e12,
                                               "bound": "tensor (tf32, three MMAs per product)",
                                               "executed_tflops": exec_flops / t / 1e12,
                                               "peak_tflops": tf32_peak, "frac": exec_flops / t / 1e12 / tf32_peak,
                                               "peak_source": src + " bf16 x nominal tf32/bf16 ratio"}
    log("loss fwd", res["pair_loss_fwd_10k_x_100k_512_128"])
    t = timed(lambda: lv.leanvec_ood_loss_bwd(Ai, Ai, Qo, Xo), 2)
    # the backward forms R = Qt X^T and contracts it twice (R X', R^T Q'), each in tf32x3 form:
    # 3 x 2 m n (D + 2 d) executed flops; the final d x D products (3 x 2 (m + n) d D) are not counted
    exec_bwd = 3 * 2.0 * Qo.shape[0] * Xo.shape[0] * (512 + 2 * 128)
    res["pair_loss_bwd_10k_x_100k_512_128"] = {"seconds": t, "pair_tflops": exec_bwd / 3 / t / 1e12,
                                               "bound": "tensor (tf32, three MMAs per product)",
                                               "executed_tflops": exec_bwd / t / 1e12, "peak_tflops": tf32_peak,
                                               "frac": exec_bwd / t / 1e12 / tf32_peak,
                                               "peak_source": src + " bf16 x nominal tf32/bf16 ratio"}
    log("loss bwd", res["pair_loss_bwd_10k_x_100k_512_128"])
    out = {"metric": "offline / auxiliary kernels through the C ABI: seconds per call and the fraction of each "
                     "kernel's roofline (tensor: bf16 peak " + src + ", fp8 = 2x bf16; hbm: copy peak " + hbm_src + ")",
           "workload": f"id-{n // 1000}k-{D} (anisotropic mixture, unit norm), d = {d}; OOD fits on 100k x 512 "
                       f"database samples and 10k learning queries, d = 128",
           "results": res, "data": "synthetic"}
    print(json.dumps(out), flush=True)


def bench_samples(args, dev):
    """Sample sizes of the fit (the paper's appendix study): on the ood-1M-512 workload, the
    second moments, the LeanVec-OOD projections (Frank-Wolfe A, B; eigenvector search P) and the
    LeanVec-ID projection are learned once from the full learning sets (1M database vectors,
    10k learning queries) and again from the first n_s rows of each (the rows are independent
    draws of the mixture, so these are uniform samples); reported are
    the relative Frobenius errors of n_s^-1 K and of the projectors A^T A, B^T B, P^T P against the
    full-set ones, and the exhaustive-search recall@10 of <A q, B x> on 10k held-out OOD test
    queries (ground truth: exact inner products) for each sample size."""
    from paper_2312_16335_gb300 import build_lib
    build_lib.build()
    import paper_2312_16335_gb300 as lv
    n, m, D, d = args.n, args.m, 512, 128
    X, Q, Ql = workloads.make_workload_torch("anisotropic", n, m, D, 1000, cfg=3, device=dev, ood=True, m_learn=m)
    truth = ground_truth(X, Q, 10)

    def rel(a, b):
        return float((a.double() - b.double()).norm() / b.double().norm())

    def projector(M):
        M = M.double()
        return M.T @ M

    def bf_recall(A, B):
        """recall@10 of the exhaustive search by <A q, B x> (float32 projections by the library)"""
        qa = lv.leanvec_project(Q, A)
        best_s = torch.full((Q.shape[0], 10), -float("inf"), device=dev)
        best_i = torch.full((Q.shape[0], 10), -1, dtype=torch.int64, device=dev)
        for s0 in range(0, n, 131072):
            xb = lv.leanvec_project(X[s0:s0 + 131072].contiguous(), B)
            S = qa @ xb.T
            v, i = torch.topk(S, 10, dim=1)
            cs, ci = torch.cat([best_s, v], 1), torch.cat([best_i, i + s0], 1)
            o = torch.topk(cs, 10, dim=1)
            best_s, best_i = o.values, torch.gather(ci, 1, o.indices)
        return recall_at(best_i, truth, 10)

    def fit_all(nx, nq):
        Xs, Qs = X[:nx].contiguous(), Ql[:nq].contiguous()  # rows are i.i.d. draws: the first rows are a sample
        KX = lv.leanvec_second_moment(Xs, precision=lv.PREC_BF16) / nx
        KQ = lv.leanvec_second_moment(Qs, precision=lv.PREC_BF16) / nq
        A, B, rf = lv.leanvec_fit_ood(Xs, Qs, d, method=lv.FIT_FW, precision=lv.PREC_BF16)
        P, _, re = lv.leanvec_fit_ood(Xs, Qs, d, method=lv.FIT_ES, precision=lv.PREC_BF16)
        I = lv.leanvec_fit_id(Xs, d, precision=lv.PREC_BF16)
        return dict(KX=KX, KQ=KQ, A=A, B=B, P=P, I=I, fw_iters=rf["iterations"], es_beta=re["beta"])

    t0 = time.time()
    full = fit_all(n, m)
    log(f"full-set fit {time.time() - t0:.1f}s")
    ref = {k: projector(full[k]) for k in ("A", "B", "P", "I")}
    res = {"full": {"recall_fw": bf_recall(full["A"], full["B"]), "recall_es": bf_recall(full["P"], full["P"]),
                    "recall_id": bf_recall(full["I"], full["I"]), "fw_iterations": full["fw_iters"],
                    "es_beta": full["es_beta"]}}
    log(f"full: {res['full']}")
    for ns in (D, 2 * D, 4 * D, 8 * D, 10_000, 100_000, 1_000_000):
        nx, nq = min(ns, n), min(ns, m)
        f = fit_all(nx, nq)
        r = {"n_x": nx, "n_q": nq,
             "err_KQ": rel(f["KQ"], full["KQ"]), "err_KX": rel(f["KX"], full["KX"]),
             "err_AtA": rel(projector(f["A"]), ref["A"]), "err_BtB": rel(projector(f["B"]), ref["B"]),
             "err_PtP": rel(projector(f["P"]), ref["P"]), "err_ID": rel(projector(f["I"]), ref["I"]),
             "recall_fw": bf_recall(f["A"], f["B"]), "recall_es": bf_recall(f["P"], f["P"]),
             "recall_id": bf_recall(f["I"], f["I"]), "fw_iterations": f["fw_iters"], "es_beta": f["es_beta"]}
        res[ns] = r
        log(f"n_s={ns}: {r}")
    out = {"metric": "relative Frobenius errors of the sample second moments and learned projectors, and the "
                     "exhaustive-search recall@10 of <A q, B x>, vs the learning sample size n_s",
           "workload": f"ood-{n // 1000}k-512: {m} learning + {m} held-out OOD queries, d = {d}; full sets = "
                       f"{n} database vectors and {m} learning queries; n_s rows of each (queries capped at {m})",
           "results": res, "data": "synthetic"}
    print(json.dumps(out), flush=True)


def bench_dsweep(args, dev):
    """Target-d selection on the id-1M-768 workload through the library's autotuner
    (autotune_target_d): one graph (the id workload's, see --graph), then for each primary
    dimension d the LeanVec-ID projection of that size (100k-row sample), its primaries and
    secondaries, the smallest L with recall@10 >= 0.90 (rerank = L, max_hops = ceil(c L) for
    the hop factor c) and the QPS there."""
    S = setup(args, dev, with_base=False)
    lv, X, Q, truth = S["lv"], S["X"], S["Q"], S["truth"]
    graph, entry = S["graph"], S["entry"]
    del S["idx"]
    sub = torch.from_numpy(workloads.subsample_rows(args.n, min(args.n, 100_000), cfg=2)).to(dev)
    Xs = X.index_select(0, sub).contiguous()
    proj = lv.PREC_BF16 if args.projection == "bf16" else lv.PREC_FP32

    def fit(_, d):
        P = lv.leanvec_fit_id(Xs, d)
        return P, P

    tune = lv.autotune_target_d(X, Q, truth, graph, entry, ds=(64, 96, 128, 160, 192, 224, 240), k=10,
                                target=TARGET, L_grid=tuple(L_GRID), fit=fit, width=args.width, projection=proj,
                                hop_factor=args.hop_factor)
    res = {r["d"]: {k: v for k, v in r.items() if k != "A"} for r in tune["table"]}
    for d, r in res.items():
        log(f"d={d}: {r}")
    best = tune["best"]["d"] if tune["best"] else None
    out = {"metric": "QPS at 10-recall@10 = 0.90 vs the primary dimension d (one graph, built on "
                     + ("full-D LVQ-8 codes)" if args.graph == "full" else "the d = 160 primaries)"),
           "workload": f"id-{args.n // 1000}k-{args.D}, {args.m} ID queries, LeanVec-ID LVQ-8 primaries of d dims "
                       f"+ LVQ-8 secondaries, width {args.width}, {args.projection} projection, "
                       f"max_hops = ceil({args.hop_factor} L)",
           "results": res, "best_d": best, "data": "synthetic"}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=0, help="database size (default: the workload's, 1M or 10M)")
    ap.add_argument("--m", type=int, default=0, help="queries (default: the workload's, 10k / 50k / 100k)")
    ap.add_argument("--D", type=int, default=768)
    ap.add_argument("--d", type=int, default=160)
    ap.add_argument("--components", type=int, default=1000)
    ap.add_argument("--R", type=int, default=64)
    ap.add_argument("--L_build", type=int, default=128)
    ap.add_argument("--alpha", type=float, default=None,
                    help="RobustPrune alpha (default 1.02; 1.2 for the l2 workload)")
    ap.add_argument("--secondary", default="lvq8", choices=["lvq8", "fp16"],
                    help="id workload: LVQ-8 secondaries (the configured encoding) or FP16 ones (the paper's "
                         "default in its experiments)")
    ap.add_argument("--graph", default="full", choices=["full", "primary"],
                    help="id and precision workloads: build the searched graph on LVQ-8 codes of the unreduced "
                         "vectors (full, the paper's setting for its search comparisons) or on the d-dim primaries")
    ap.add_argument("--rule", type=int, default=None,
                    help="RobustPrune rule: 0 alpha-scaled similarity, 1 Vamana's L2 rule on unit-norm vectors "
                         "(default 1; 0 for the l2 workload, whose build scores are negative squared distances)")
    ap.add_argument("--batch", type=int, default=None,
                    help="build batch (default 65536; 16384 for the l2 workload, whose 992-byte records leave "
                         "room for a smaller reverse-edge pool per target)")
    ap.add_argument("--L", type=int, default=0, help="fixed beam width (skips the recall sweep)")
    ap.add_argument("--max-hops", type=int, default=0, help="expansion budget with --L (0: none)")
    ap.add_argument("--hop-factor", type=float, default=1.0,
                    help="id workload: expansion budget max_hops = ceil(c L) for hop factor c (0 = no budget); "
                         "both arms, L calibrated for recall 0.90 under it")
    ap.add_argument("--hop-sweep", action="store_true",
                    help="id workload: calibrate every hop factor of %s and keep the fastest (both arms)"
                         % (HOP_FACTORS,))
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--hash", type=int, default=0, help="visited-cache slots per query (0 = library default)")
    ap.add_argument("--width", type=int, default=2, help="search width (beam members expanded per round)")
    ap.add_argument("--queries-per-warp", dest="qpw", type=int, default=0, choices=[0, 1, 2],
                    help="queries per warp of the beam kernel (0 = the library default, 1)")
    ap.add_argument("--visited-bits", dest="vbits", type=int, default=0, choices=[0, 16, 32],
                    help="visited-cache slot width: 32-bit ids (0 = the library default) or 16-bit tags")
    ap.add_argument("--projection", default="bf16", choices=["fp32", "bf16"],
                    help="query projection GEMM: bf16 tcgen05 tensor cores or fp32 CUDA cores")
    ap.add_argument("--workload", default="id", choices=["id", "c1", "ood", "uneven", "precision", "dsweep",
                                                      "buildstudy", "l2", "kernels", "samples", "loss"],
                    help="id: the headline 1M x 768 ID workload; c1: the L2-resident 10k x 128 ID configuration; ood: the shifted-query 1M x 512 comparison; "
                         "uneven: 10M x 200 mixed-k / mixed-L batch in one CUDA-graph launch; "
                         "precision: 10M x 768 with FP8 projection and LVQ-4 primaries; "
                         "dsweep: QPS at recall 0.90 vs the primary dimension d on the id workload's graph; "
                         "buildstudy: graph build on primaries vs on full-D LVQ-8 codes; "
                         "l2: Euclidean 1M x 960 (gist-960-1M shape), LeanVec vs FP32 at recall 0.90; "
                         "kernels: the offline / auxiliary kernels alone against their rooflines; "
                         "samples: fit sample-size study (second moments, projectors, exhaustive-search recall); "
                         "loss: the pair loss forward / backward of the differentiation form alone")
    ap.add_argument("--tune-d", action="store_true",
                    help="uneven workload: the code width d by the autotuner on a full-D graph, and the uneven "
                         "batch at the configured and the tuned d")
    ap.add_argument("--diagnose", action="store_true",
                    help="precision workload: where recall is lost (exhaustive primary ceiling, full-D graph)")
    ap.add_argument("--grad-steps", type=int, default=100, help="ood workload: Adam steps of the gradient optimiser")
    ap.add_argument("--grad-lr", type=float, default=1e-4,
                    help="ood workload: Adam learning rate (at D = 512 the projected iteration is unstable above "
                         "about 3e-4; the best iterate is kept)")
    ap.add_argument("--profile", action="store_true",
                    help="setup, then only `steps` searches at --L inside an NVTX range 'timed' (for ncu)")
    args = ap.parse_args()
    # the id workload calibrates the expansion budget per arm (the fastest hop factor whose
    # smallest L reaches recall 0.90) unless a factor is given
    if args.workload == "id" and "--hop-factor" not in sys.argv:
        args.hop_sweep = True
    sizes = {"id": (1_000_000, 10_000), "c1": (10_000, 1000), "ood": (1_000_000, 10_000), "uneven": (10_000_000, 50_000),
             "precision": (10_000_000, 100_000), "dsweep": (1_000_000, 10_000),
             "buildstudy": (1_000_000, 10_000), "l2": (1_000_000, 10_000),
             "kernels": (1_000_000, 10_000), "samples": (1_000_000, 10_000), "loss": (100_000, 10_000)}[args.workload]
    args.n = args.n or sizes[0]
    args.m = args.m or sizes[1]
    l2 = args.workload == "l2"
    if args.alpha is None:
        args.alpha = 1.2 if l2 else 1.02
    if args.rule is None:
        args.rule = 0 if l2 else 1
    if args.batch is None:
        args.batch = 16384 if l2 else 65536
    if l2 and "--D" not in sys.argv:
        args.D = 960

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if args.workload == "c1":
        bench_c1(args, dev)
        return
    if args.workload == "ood":
        bench_ood(args, dev)
        return
    if args.workload == "uneven":
        bench_uneven(args, dev)
        return
    if args.workload == "precision":
        bench_precision(args, dev)
        return
    if args.workload == "dsweep":
        bench_dsweep(args, dev)
        return
    if args.workload == "buildstudy":
        bench_buildstudy(args, dev)
        return
    if args.workload == "l2":
        bench_l2(args, dev)
        return
    if args.workload == "kernels":
        bench_kernels(args, dev)
        return
    if args.workload == "samples":
        bench_samples(args, dev)
        return
    if args.workload == "loss":
        bench_loss(args, dev)
        return
    workload = (f"id-{args.n // 1000}k-{args.D}: anisotropic Gaussian mixture ({args.components} components, "
                f"i^-1 spectrum), unit norm, inner product; {args.m} ID queries; LeanVec-ID d={args.d}, "
                f"LVQ-8 primary + LVQ-8 secondary; GPU-built graph R={args.R}, L_build={args.L_build}, "
                f"alpha={args.alpha} ({'unit-norm L2' if args.rule else 'alpha-scaled IP'} prune rule), built on "
                f"{'full-D LVQ-8 codes' if args.graph == 'full' else 'the primaries'}; k=10, rerank=L, "
                + ("max_hops=ceil(c L) with the hop factor c of each arm calibrated (the fastest of %s whose "
                   "smallest L reaches recall@10 0.90; 0 = no budget)" % (HOP_FACTORS,) if args.hop_sweep else
                   'max_hops=ceil(%g L)' % args.hop_factor if args.hop_factor else 'no expansion budget'))
    if args.secondary == "fp16":
        workload = workload.replace("LVQ-8 primary + LVQ-8 secondary", "LVQ-8 primary + FP16 secondary")
    metric = "QPS at 10-recall@10=0.90, LeanVec vs full-D FP32 graph search; HBM GB/s"

    if args.impl == "reference":
        if rank != 0:
            return
        S = setup(args, dev, with_base=False)
        proj = S["lv"].PREC_BF16 if args.projection == "bf16" else S["lv"].PREC_FP32
        L, mh, _, table = choose_config(args, S, proj)
        vals = []
        cb = None
        O = oracle_prepare(S)
        for i in range(args.warmup + args.steps):
            r = cpu_oracle_sample(O, L, budget_s=max(2.0, args.cpu_budget / max(1, args.steps)), max_hops=mh,
                                  width=args.width)
            if i >= args.warmup:
                vals.append(r["value"])
                cb = r
        v = statistics.median(vals)
        cb["value"] = v
        out = {"impl": "reference", "metric": metric, "value": v, "unit": "queries/s", "n_gpus": 1,
               "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f64", "data": "synthetic",
               "config": id_config(args, workload, S["Q"].shape[0], L, mh, best_hop_factor(table, args.hop_factor),
                                   S["idx"].info()),
               "impl_note": "CPU oracle on the host cores (the same graph, stores and queries; the projection's "
                            "bf16 operand rounding applied in FP64)",
               "cpu_baseline": cb, "e2e": {"value": v, "unit": "queries/s", "h2d_bytes_per_step": 0,
                                             "d2h_bytes_per_step": 0}}
        print(json.dumps(out), flush=True)
        return

    S = setup(args, dev, with_base=not args.profile)
    lv, idx, base, Q, A, truth = S["lv"], S["idx"], S["base"], S["Q"], S["A"], S["truth"]
    proj = lv.PREC_BF16 if args.projection == "bf16" else lv.PREC_FP32
    m = Q.shape[0]
    k = 10
    if args.profile:
        L = args.L or 64
        for _ in range(args.warmup):
            idx.search(Q, A, k=k, L=L, rerank=L, max_hops=args.max_hops, width=args.width, hash_slots=args.hash, queries_per_warp=args.qpw, visited_bits=args.vbits,
                       projection=proj)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("timed")
        for _ in range(args.steps):
            idx.search(Q, A, k=k, L=L, rerank=L, max_hops=args.max_hops, width=args.width, hash_slots=args.hash, queries_per_warp=args.qpw, visited_bits=args.vbits,
                       projection=proj)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        print(json.dumps({"profile": True, "L": L, "max_hops": args.max_hops, "n": args.n, "m": m,
                          "steps": args.steps}), flush=True)
        return
    ids_buf = torch.empty((m, k), dtype=torch.int32, device=dev)
    sc_buf = torch.empty((m, k), dtype=torch.float32, device=dev)

    # -- choose L (and the expansion budget) for recall 0.90 (untimed)
    def lv_search(L, mh, **kw):
        return idx.search(Q, A, k=k, L=L, rerank=L, max_hops=mh, width=args.width, hash_slots=args.hash, queries_per_warp=args.qpw, visited_bits=args.vbits,
                          projection=proj, **kw)

    def base_search(L, mh, **kw):
        return base.search(Q, None, k=k, L=L, max_hops=mh, width=args.width, **kw)

    L, mh, rec, hop_table = choose_config(args, S, proj)
    factors = HOP_FACTORS if args.hop_sweep else (args.hop_factor,)
    Lb, mhb, rec_b, hop_table_b = calibrate_budget(lambda L, mh: base_search(L, mh)[0], qps_of(base_search, m),
                                                   truth, k, factors)
    if Lb is None:
        Lb, mhb = L_GRID[-1], 0
        rec_b = recall_at(base_search(Lb, mhb)[0], truth, k)
    log(f"LeanVec L={L} max_hops={mh} recall={rec:.4f}  table={hop_table}")
    log(f"FP32   L={Lb} max_hops={mhb} recall={rec_b:.4f}  table={hop_table_b}")

    # -- per-query work (untimed run with the kernel's counters)
    _, _, st = lv_search(L, mh, stats=True)
    launches = idx.info()["last_search_kernels"]
    hops = float(st[:, 0].double().mean())
    scored_gpu = float(st[:, 1].double().mean())
    inf = idx.info()

    def step(ev):
        lv_search(L, mh, out=(ids_buf, sc_buf), events=ev)

    if world > 1:
        torch.distributed.barrier()
    with Clocks(local) as clk:
        total_ms, kern_ms = time_steps(step, args.steps, args.warmup, events=True)
    ck = clk.summary()
    qps, total_ms = replica_throughput(total_ms, m, args.steps, dev)
    kern_avg = statistics.mean(kern_ms)
    hbm_peak, peak_kind = peaks()

    # -- end to end through the C ABI with host buffers: one leanvec_search_host call over
    # e2e_steps batches of the m queries (pinned host memory), each batch copied in, searched and
    # its results copied out, the copies of neighbouring batches overlapping the searches
    e2e_steps = max(5, args.steps // 2)
    Qh = Q.cpu().repeat(e2e_steps, 1).pin_memory()
    ids_h = torch.empty((m * e2e_steps, k), dtype=torch.int32).pin_memory()
    sc_h = torch.empty((m * e2e_steps, k), dtype=torch.float32).pin_memory()
    host_kw = dict(k=k, L=L, rerank=L, max_hops=mh, width=args.width, hash_slots=args.hash, queries_per_warp=args.qpw, visited_bits=args.vbits, projection=proj,
                   batch=m)
    idx.search_host(Qh[:2 * m], A, out=(ids_h[:2 * m], sc_h[:2 * m]), **host_kw)  # slots sized, streams made
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    idx.search_host(Qh, A, out=(ids_h, sc_h), **host_kw)
    e1.record()
    torch.cuda.synchronize()
    e2e_qps = m * e2e_steps / (e0.elapsed_time(e1) / 1e3)
    e2e_ok = bool((ids_h[-m:].to(dev) == ids_buf).all())  # the host results equal the device-timed step's

    # -- full-dimensional float32 baseline on the same graph
    ids_b = torch.empty((m, k), dtype=torch.int32, device=dev)
    sc_b = torch.empty((m, k), dtype=torch.float32, device=dev)
    base_ms, _ = time_steps(lambda ev: base_search(Lb, mhb, out=(ids_b, sc_b)), max(5, args.steps // 2), 2)
    qps_b = m * max(5, args.steps // 2) / (base_ms / 1e3)
    _, _, stb = base_search(Lb, mhb, stats=True)
    bytes_b = args.D * 4 + float(stb[:, 0].double().mean()) * (4 * inf["R"] + 4) + \
        float(stb[:, 1].double().mean()) * lv.leanvec_record_stride(args.D, 32)

    if rank != 0:
        return
    # -- the CPU oracle on this host's cores (bounded sample), which also gives the method's own
    # count of scored nodes per query (an exact visited set, the projection's operand rounding
    # applied), the count the algorithmic bytes use
    import oracle
    O = oracle_prepare(S, args.projection)
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        try:
            cpu = cpu_oracle_sample(O, L, args.cpu_budget, max_hops=mh, width=args.width)
        except Exception as e:  # the GPU result stands without the CPU leg
            cpu = {"error": repr(e)}
    if cpu and "scored_per_query" in cpu:
        scored_method, hops_method, method_sample = cpu["scored_per_query"], cpu["hops_per_query"], cpu["sample"]
    else:
        ms = min(m, 1000)
        r = oracle.search(O["g"], O["entry"], O["qp"][:ms], k=k, L=L, rerank=L, prim=O["prim"], sec=O["sec"],
                          qs=O["Qh"][:ms], max_hops=mh, width=args.width)
        scored_method, hops_method = float(r["scored"].mean()), float(r["hops"].mean())
        method_sample = f"first {ms} queries"
    bytes_q = method_bytes_per_query(args.D, inf["d"], 8, inf["R"], hops_method, scored_method, L)
    achieved = bytes_q * m / (kern_avg / 1e3) / 1e9
    out = {
        "metric": metric, "value": qps, "unit": "queries/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 (u8 LVQ codes decoded to f32)",
        "data": "synthetic",
        "config": id_config(args, workload, m, L, mh, best_hop_factor(hop_table, args.hop_factor), inf),
        "recall_at_10": rec, "hop_budget_table": hop_table,
        "setup_seconds": {"build": S["t_build"], "fit": S["t_fit"], "encode": S["t_enc"]},
        "e2e": {"value": e2e_qps, "unit": "queries/s", "h2d_bytes_per_step": m * args.D * 4,
                "d2h_bytes_per_step": m * k * 8, "api": "leanvec_search_host (C ABI): one call over %d batches of "
                "the %d queries in pinned host memory, each batch copied in, searched and its ids and scores "
                "copied out, the copies of neighbouring batches overlapping the searches" % (e2e_steps, m),
                "results_match_device": e2e_ok},
        # per step, as the library counts them: the projection (bf16: cast of A + the float32-input
        # GEMM), then the beam and rerank kernels of each sub-batch
        "gpu_launches": launches * args.steps,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved / hbm_peak, "traffic": recorded_traffic(args, L, mh),
                     "kernel": ("beam_half_kernel<3,8>" if args.qpw == 2 else "beam_kernel<LvqIntScorer<3,8>,search>")
                               + " + rerank_kernel",
                     "kernel_ms": kern_avg, "bytes_per_query": bytes_q,
                     "bytes_model": "4 D + hops (4 R + 4) + scored x %d + rerank x (D + 8)" %
                                    (-(-(inf["d"] + 8) // 32) * 32),
                     "hops_per_query": hops_method, "scored_per_query": scored_method,
                     "scored_counted_by": "the oracle's exact visited set (%s)" % method_sample,
                     "gpu_scored_per_query": scored_gpu, "gpu_hops_per_query": hops,
                     "gpu_rescored_bytes_per_query": max(0.0, scored_gpu - scored_method) *
                                                     (-(-(inf["d"] + 8) // 32) * 32),
                     "peak_kind": peak_kind},
        "baseline_fp32": {"value": qps_b, "unit": "queries/s", "L": Lb, "max_hops": mhb, "recall_at_10": rec_b,
                          "hop_factor": best_hop_factor(hop_table_b, None),
                          "hop_budget_table": hop_table_b, "bytes_per_query": bytes_b,
                          "speedup_leanvec": qps / world / qps_b},
        "cpu_baseline": cpu,
        "clocks": ck,
    }

    def interp(table, Lc, mhc):
        row = [t for t in table if t.get("L") == Lc and t.get("max_hops") == mhc and t.get("qps")]
        return row[0].get("qps_interpolated") if row else None

    if hop_table and hop_table_b:
        out["qps_at_0.90_interpolated"] = {
            "leanvec": interp(hop_table, L, mh), "fp32": interp(hop_table_b, Lb, mhb),
            "rule": "log QPS linear in recall@10 between the grid point below 0.90 and the smallest one at or "
                    "above it, each arm at its chosen hop factor (calibration timings, 5 calls each); the "
                    "value above is the measured grid point"}
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
