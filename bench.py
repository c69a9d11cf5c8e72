#!/usr/bin/env python
"""Benchmark of the fused FUnc-SNE iteration on GB300.

Workload: the 1M-point spectrum workload (N=1,000,000, D=50 FP32, feature
variance ~1/j over 50 anisotropic Zipf-sized clusters; d=16, k_hd=32,
k_ld=32, n_neg=32, alpha=1, perplexity 30; synthetic, seed 0). One step =
one full iteration: HD refinement (forced every iteration), bandwidth
bisection for flagged points, LD refinement, attraction / repulsion /
normalisation, momentum update. Metric: iterations/s, BF16 HD storage vs
FP32 at equal KNN recall (the FP32 re-rank makes the neighbour sets equal).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun) every rank runs an independent replica of the
workload ("replicas only": the iteration has no cross-GPU step here).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "iters/s at N=1M (KNN refine+gradient), BF16 vs FP32 at equal KNN recall"
UNIT = "iter/s"
WORKLOAD = "spectrum-1m"
BURN_IN = 200          # untimed iterations after set-up, so lists are near steady state
RECALL_QUERIES = 1000  # sampled queries for HD-KNN recall against brute force
FALLBACK_HBM_GBS = 6800.0


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def algorithmic_bytes_per_point(D, d, k_hd, k_ld, n_neg, row_bytes, rerank_rows=0.0):
    """Minimum bytes one point moves in each kernel of one iteration (HD
    refinement forced), before sector rounding. the design doc derives them."""
    y = 4 * d
    hd = ((1 + 32) * row_bytes + rerank_rows * 4 * D   # own row, candidate rows, exact re-ranks
          + 8 * k_hd + 4 * k_ld                        # HD list (index, d2) and LD list of t
          + 20 * 4                                     # neighbour-of-neighbour index reads
          + 8 * k_hd)                                  # HD list of t+1
    ld = (4 * k_ld + 4 * k_hd + 16 * 4                 # LD and HD lists of t, index reads
          + (1 + k_ld + 32) * y                        # own, old-list and candidate rows of Y_t
          + 4 * k_ld)                                  # LD list of t+1
    forces = (8 * k_hd + 4 * k_ld                      # HD list and P, LD list of t+1
              + (1 + k_hd + k_ld + n_neg) * y          # own row and gathered rows of Y_t
              + k_hd * y + 2 * y)                      # reverse attraction (scatter), A_i and R_i
    update = 7 * y                                     # Y, V, A read+write, R read
    return {"hd_refine": hd, "ld_refine": ld, "forces": forces, "update": update}


def kernel_source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2509_07681_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(f.encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def committed_traffic(kernel_hash, precision, kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, valid
    only for the kernel sources it was captured from."""
    path = os.path.join(ROOT, "profiles", "kernels_spectrum-1m.json")
    try:
        with open(path) as f:
            js = json.load(f)
    except Exception:
        return None
    if js.get("kernel_hash") != kernel_hash:
        return None
    ent = js.get("dram_bytes_per_launch", {}).get(precision, {}).get(kernel)
    return float(ent) if ent is not None else None


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        if not self.rows:
            return None
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(self.rows)}


def run_ours(args, rank, world):
    import torch
    from paper_2509_07681_gb300 import funcsne as F
    from paper_2509_07681_gb300 import synth
    from paper_2509_07681_gb300.build import build

    local = _env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    build()
    F.load()
    X, p = synth.make(WORKLOAD, n=args.n)
    N, D = X.shape
    K, W = args.steps, args.warmup
    stream = torch.cuda.Stream()

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    m = F.FuncSNE(X, p["d"], p["k_hd"], p["k_ld"], p["n_neg"], p["alpha"], p["perplexity"], seed=0)
    m.set_stream(stream)
    m.set_option("hd_mode", 1)
    m.step(BURN_IN)
    m.sync()
    base = m.export_state()

    results = {}
    clocks = ClockSampler(local)
    precisions = [("fp32", F.FP32), ("bf16", F.BF16), ("fp8", F.FP8)]
    for name, prec in precisions:
        m.import_state(base)
        m.set_option("precision", prec)
        m.set_option("hd_mode", 1)
        m.step(W)
        m.sync()
        st_w = m.export_state()
        s0 = m.stats()
        barrier()
        if name == "fp32":
            clocks.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        m.step(K)
        e1.record(stream)
        barrier()
        total_ms = e0.elapsed_time(e1)
        s1 = m.stats()
        m.sync()
        if dist is not None:
            t = torch.tensor([total_ms], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            total_ms = float(t.item())
        # per-kernel device times: the same iterations again with events
        # between the kernels (sequential launches), from the same state
        m.import_state(st_w)
        kms = m.profile_step(K)
        m.sync()
        scored = s1["cand_scored"] - s0["cand_scored"]
        rer = s1["cand_reranked"] - s0["cand_reranked"]
        results[name] = dict(total_ms=total_ms, kernel_ms={k: v / K for k, v in kms.items()},
                             rerank_rows=(rer / (N * K)) if prec != F.FP32 else 0.0,
                             rerank_frac=(rer / scored) if scored else None,
                             hd_idx=m.knn(F.SPACE_HD, with_d2=False))
    clk = clocks.stop()

    # KNN recall of each precision's lists against brute force on sampled queries
    rng = np.random.default_rng(0)
    q = np.sort(rng.choice(N, size=min(RECALL_QUERIES, N), replace=False)).astype(np.int32)
    exact, _ = m.exact_knn(q, p["k_hd"])
    from paper_2509_07681_gb300.quality import recall
    for name in results:
        results[name]["recall"] = recall(results[name]["hd_idx"][q], exact)
        results[name]["sets_equal_fp32"] = bool(np.array_equal(results[name]["hd_idx"], results["fp32"]["hd_idx"]))

    # end to end through the C ABI with host buffers: create from pinned host
    # X (H2D), then every step read the embedding back to pinned host memory
    m.close()
    Xp = torch.from_numpy(X).pin_memory()
    Yp = torch.empty((N, p["d"]), dtype=torch.float32).pin_memory()
    barrier()
    t0 = time.perf_counter()
    m2 = F.FuncSNE(Xp, p["d"], p["k_hd"], p["k_ld"], p["n_neg"], p["alpha"], p["perplexity"], seed=0,
                   hd_mode=1, precision=F.BF16)
    for _ in range(K):
        m2.step(1)
        m2.embedding(out=Yp)
    m2.sync()
    e2e_s = time.perf_counter() - t0
    m2.close()
    if dist is not None:
        t = torch.tensor([e2e_s], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return None
    head = results["bf16"]
    value = world * K / (head["total_ms"] / 1e3)
    peak, peak_kind = measured_peaks()
    khash = kernel_source_hash()
    row_bytes = {"fp32": 4 * D, "bf16": 2 * D + 4, "fp8": D + 4}
    for name in results:
        r = results[name]
        per = algorithmic_bytes_per_point(D, p["d"], p["k_hd"], p["k_ld"], p["n_neg"], row_bytes[name],
                                          r["rerank_rows"])
        r["alg_bytes"] = {k: N * v for k, v in per.items()}
        r["achieved_gbs"] = {k: r["alg_bytes"][k] / (r["kernel_ms"][k] / 1e3) / 1e9 for k in per}
    top = max(head["kernel_ms"], key=head["kernel_ms"].get)
    traffic = committed_traffic(khash, "bf16", top)
    roofline = {"bound": "hbm", "achieved": round(head["achieved_gbs"][top], 1), "peak": peak, "unit": "GB/s",
                "frac": round(head["achieved_gbs"][top] / peak, 4), "traffic": traffic,
                "kernel": f"{top} (BF16 rows)", "peak_source": peak_kind,
                "alg_bytes_per_launch": int(head["alg_bytes"][top]),
                "step_frac": round(sum(head["alg_bytes"].values()) / (head["total_ms"] / K / 1e3) / 1e9 / peak, 4)}
    cpu = cpu_baseline(args, X, p, sample_n=100000, steps=2) if world == 1 else None
    line = {
        "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": round(head["total_ms"] / K, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "N": N, "D": D, "d": p["d"], "k_hd": p["k_hd"], "k_ld": p["k_ld"],
                   "n_neg": p["n_neg"], "alpha": p["alpha"], "perplexity": p["perplexity"],
                   "hd_refine": "every iteration", "storage": "bf16 rows + fp32 boundary re-rank",
                   "burn_in": BURN_IN, "l2": "working set > L2 (X 208 MB + lists 768 MB)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "precisions": {n: {"iters_per_s": round(K / (r["total_ms"] / 1e3), 2),
                           "kernel_ms": {k: round(v, 4) for k, v in r["kernel_ms"].items()},
                           "recall_at_k_hd": round(r["recall"], 5), "sets_equal_fp32": r["sets_equal_fp32"],
                           "rerank_rows_per_point": round(r["rerank_rows"], 3),
                           "rerank_fraction": None if r["rerank_frac"] is None else round(r["rerank_frac"], 4),
                           "achieved_alg_gbs": {k: round(v, 1) for k, v in r["achieved_gbs"].items()}}
                       for n, r in results.items()},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": {"value": round(world * K / e2e_s, 3), "unit": UNIT, "h2d_bytes_per_step": int(X.nbytes / K),
                "d2h_bytes_per_step": int(N * p["d"] * 4),
                "note": "create from pinned host X (H2D, init) + K x (step + embedding read-back), BF16"},
        "gpu_launches": 4 * K * len(results),
        "clocks": clk,
        "kernel_hash": khash,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return line


def cpu_baseline(args, X, p, sample_n=None, steps=1):
    """The FP64 oracle, as it stands, on the host cores: a bounded sample of the
    workload (the same generator at N=sample_n), one timed iteration after its
    own initialisation, scaled linearly to N=1M (the iteration is O(N))."""
    import oracle as O
    from paper_2509_07681_gb300 import synth

    n = sample_n or args.cpu_sample
    Xs, _ = synth.make(WORKLOAD, n=n)
    o = O.OracleState(Xs, p["d"], p["k_hd"], p["k_ld"], p["n_neg"], p["alpha"], p["perplexity"], seed=0,
                      hd_mode=1)
    t0 = time.perf_counter()
    for _ in range(steps):
        o.step()
    dt = (time.perf_counter() - t0) / steps
    scale = X.shape[0] / n
    return {"value": round(1.0 / (dt * scale), 6), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{WORKLOAD} generator at N={n} (same D, d, k, n_neg), {steps} oracle iteration(s) "
                      f"after its own init, {dt:.2f} s/iter scaled x{scale:.0f} to N={X.shape[0]}"}


def run_reference(args, rank, world):
    """The oracle on the host cores as the reference arm (rank 0 only)."""
    if rank != 0:
        return None
    import oracle as O
    from oracle.build import build_oracle
    from paper_2509_07681_gb300 import synth

    build_oracle()
    Xfull_n = 1_000_000 if args.n is None else args.n
    n = args.cpu_sample
    Xs, p = synth.make(WORKLOAD, n=n)
    o = O.OracleState(Xs, p["d"], p["k_hd"], p["k_ld"], p["n_neg"], p["alpha"], p["perplexity"], seed=0, hd_mode=1)
    for _ in range(args.warmup):
        o.step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.step()
    dt = (time.perf_counter() - t0) / args.steps
    scale = Xfull_n / n
    value = 1.0 / (dt * scale)
    sample = (f"{WORKLOAD} generator at N={n}, {args.steps} timed oracle iterations after {args.warmup} "
              f"warm-up, {dt:.3f} s/iter scaled x{scale:.0f} to N={Xfull_n}")
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * scale * 1e3, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "N": Xfull_n, "hd_refine": "every iteration"},
            "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return line


def run_profile_case(args):
    """A short, fixed sequence of launches for ncu: create the workload at N
    (default 1M), then for each precision `warmup` + `steps` iterations with
    HD refinement every iteration. Prints one line per precision."""
    from paper_2509_07681_gb300 import funcsne as F
    from paper_2509_07681_gb300 import synth
    from paper_2509_07681_gb300.build import build

    build()
    X, p = synth.make(WORKLOAD, n=args.n)
    m = F.FuncSNE(X, p["d"], p["k_hd"], p["k_ld"], p["n_neg"], p["alpha"], p["perplexity"], seed=0)
    m.set_option("hd_mode", 1)
    if args.burn_in:
        m.step(args.burn_in)
        m.sync()
    for name in args.precisions.split(","):
        m.set_option("precision", {"fp32": F.FP32, "bf16": F.BF16, "fp8": F.FP8}[name])
        m.profile_step(args.warmup)
        kms = m.profile_step(args.steps)
        m.sync()
        print(f"{name}: N={X.shape[0]} " + " ".join(f"{k} {v / args.steps:.4f} ms" for k, v in kms.items()),
              flush=True)
    m.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=None, help="override N (default: the workload's 1,000,000)")
    ap.add_argument("--cpu-sample", type=int, default=20000, help="points in the CPU oracle sample")
    ap.add_argument("--mode", choices=["bench", "ncu"], default="bench",
                    help="ncu: the short fixed launch sequence used for profiling")
    ap.add_argument("--precisions", default="fp32,bf16,fp8", help="precisions of --mode ncu")
    ap.add_argument("--burn-in", type=int, default=0, help="--mode ncu: untimed iterations first")
    args = ap.parse_args()
    if args.mode == "ncu":
        run_profile_case(args)
        return
    if args.warmup < 3:
        args.warmup = 3
    rank = _env_int("RANK", 0)
    world = _env_int("WORLD_SIZE", 1)
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world)


if __name__ == "__main__":
    main()
