"""Benchmark of the index-mapping hot path on the GPU (one JSON line).

Workload: the single large launch -- 1024 x 1024 x 512 points (2^29) on a
machine of 64 nodes x 8 processors, a seeded random split/merge/swap chain of
depth 4, in its three variants (block, cyclic, block-cyclic(4)), 7-point
stencil with 8-byte elements.  One step maps every point of the three
variants (int32 ids, per-processor histogram) and reduces the halo volume
(total and per-processor received bytes): 3 x 2^29 points per step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Metric: points mapped per second (whole job, all ranks).  Each rank maps its
own copy of the launch (replicas, weak scaling); there is no data-path
collective.  --impl reference times the CPU oracle on a bounded sample of the
same launch on the host cores.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2507_17087_gb300 import workloads as W  # noqa: E402

METRIC = "points mapped/s"
UNIT = "points/s"
VARIANTS = ("block", "cyclic", "block_cyclic")
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one full-size
# id-writer launch, from a separate ncu capture of this kernel (not measured
# in this run; None once the kernel changes, until it is captured again).
K_IDS_TRAFFIC_BYTES = 2086498560 + 46080


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=600)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=4)
    ap.add_argument("--cpu-sample", type=int, default=1 << 25,
                    help="points of the launch the CPU oracle maps for cpu_baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the search / batched / learned measurements")
    ap.add_argument("--profile-case", choices=sorted(PROFILE_CASES),
                    help="run one small case for a profiler capture and exit (no JSON line)")
    return ap.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(names, parts[3:7]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def launches():
    out = []
    for v in VARIANTS:
        cfg = W.large_config(v)
        out.append(cfg)
    return out


def cpu_baseline(sample: int, single_core: bool = True):
    """The CPU oracle, as it stands, on the first `sample` points of the block
    variant: owner of each point and of its neighbours (ids + halo)."""
    import oracle as O
    cfg = W.large_config("block")
    chain = O.chain_from_draws(*cfg["machine"], cfg["draws"])
    ref = O.Launch(cfg["L"], cfg["machine"], chain, cfg["dist"])
    cores = os.cpu_count() or 1
    ref.map_range(cfg["face"], 0, 4096, threads=1)   # warm the library
    t0 = time.perf_counter()
    ref.map_range(cfg["face"], 0, sample, threads=cores)
    dt = time.perf_counter() - t0
    res = {"value": sample / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"first {sample} points of the 1024x1024x512 block launch: owner of each point "
                     f"and of its 6 neighbours (ids + halo), std::thread over {cores} cores",
           "seconds": dt}
    if not single_core:
        return res
    # one core, on a sample of the same points as many times smaller as there
    # are cores
    s1 = max(4096, sample // cores)
    t0 = time.perf_counter()
    ref.map_range(cfg["face"], 0, s1, threads=1)
    dt1 = time.perf_counter() - t0
    res["single_core"] = {"value": s1 / dt1, "unit": UNIT, "sample": f"first {s1} points, one thread",
                          "seconds": dt1}
    return res


def extra_search(N, W, torch):
    """Exact candidates/s of the exhaustive decompose search (every candidate's
    secondary scanned) and the time to the optimum with the primary bound."""
    qs = [q for q in W.search_queries(16) if q["machine"][0] * q["machine"][1] in (2520, 3600)][:2]
    N.decompose_search(qs[:1], full=True)   # warm
    out = []
    for q in qs:
        N.decompose_search([q])   # untimed: builds the candidate space once
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = N.decompose_search([q], full=True)[0]
        t_full = time.perf_counter() - t0
        t0 = time.perf_counter()
        r2 = N.decompose_search([q])[0]
        t_bound = time.perf_counter() - t0
        assert r2["index"] == r["index"]
        out.append({"MNK": q["MNK"], "P": q["machine"][0] * q["machine"][1], "candidates": r["n_candidates"],
                    "ms_full": 1e3 * t_full, "ms_primary_bound": 1e3 * t_bound})
    cands = sum(o["candidates"] for o in out)
    secs = sum(o["ms_full"] for o in out) / 1e3
    return {"metric": "exact candidates/s", "value": cands / secs, "unit": "candidates/s",
            "workload": "3-D matmul decompose search, all ordered 3-factorisations x chains of depth <= 3, "
                        "every candidate's moved-tile cost evaluated", "queries": out}


def extra_batched(N, W, torch, dev, runs=5):
    """The 10,000-query batch in one graph replay."""
    qs = W.batched_queries(10000)
    launches = [(q["L"], q["machine"], N.chain_from_draws(*q["machine"], q["draws"]), q["dist"], q["face"])
                for q in qs]
    t0 = time.perf_counter()
    b = N.Batch(launches)
    t_create = time.perf_counter() - t0
    info = b.info()
    ids = torch.empty(int(info["total_ids"]), dtype=torch.int32, device=dev)
    hist = torch.empty(int(info["total_procs"]), dtype=torch.int64, device=dev)
    recv = torch.empty(int(info["total_procs"]), dtype=torch.int64, device=dev)
    halo = torch.empty(b.n, dtype=torch.int64, device=dev)
    b.run(ids=ids, hist=hist, halo=halo, recv=recv, autotune=True)
    b.run(ids=ids, hist=hist, halo=halo, recv=recv)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(runs):
        b.run(ids=ids, hist=hist, halo=halo, recv=recv)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / runs
    points = sum(math.prod(q["L"]) for q in qs)
    res = {"metric": "points mapped/s", "value": points / (ms / 1e3), "unit": "points/s", "queries": len(qs),
           "points": points, "ms_per_batch": ms, "ms_plan_once": 1e3 * t_create,
           "tile_groups": b.info()["tile_groups"], "hbm_gbs_ids": 4 * points / (ms / 1e3) / 1e9}
    b.close()
    del ids, hist, recv, halo
    torch.cuda.empty_cache()
    return res


def extra_learned(N, W, torch, n_train=512, per_query=4096, epochs=8, n_eval=200, n_cal=64):
    """Learned pruning: train on exact labels (three runs, the one with the
    least calibration bound kept), calibrate the margin rule on held-out
    training-distribution queries, then on 200 held-out evaluation queries
    compare time-to-optimum and regret of (a) the trained model,
    (b) the same network untrained (random initialisation, no calibration),
    (c) the no-network exact search with the primary bound and (d) the
    exhaustive search of every candidate.  Every search runs once untimed
    first (the candidate space of a machine is built once and cached)."""
    # three training runs (different seeds); the model whose calibration bound
    # on the held-out calibration queries is least is kept (selection on
    # held-out data, not on the evaluation queries)
    calq = W.search_training_queries(n_cal, first_index=40000)
    trainq = W.search_training_queries(n_train)
    model, bound, loss, bounds = None, None, None, []
    t_train = t_cal = 0.0
    for seed in (3, 4, 5):
        m = N.MLP(seed=8 + seed)
        t0 = time.perf_counter()
        l = m.train_search(trainq, samples_per_query=per_query, epochs=epochs, batch=4096, lr=1e-3, seed=seed)
        torch.cuda.synchronize()
        t_train += time.perf_counter() - t0
        t0 = time.perf_counter()
        b = m.calibrate(calq)
        t_cal += time.perf_counter() - t0
        bounds.append(b)
        if model is None or b < bound:
            if model is not None:
                model.close()
            model, bound, loss = m, b, l
        else:
            m.close()
    untrained = N.MLP(seed=99)
    evalq = W.search_queries(n_eval, first_index=9000)

    def timed(fn):
        t = time.perf_counter()
        r = fn()
        return r, time.perf_counter() - t

    arms = {"trained": model, "untrained": untrained}
    acc = {a: {"s": 0.0, "zero_regret": 0, "zero_regret_top_k_only": 0, "fallbacks": 0, "n_exact": 0,
               "accepted": {}, "regret_by_rule": {}, "phase": {"prepare": 0.0, "model": 0.0, "exact": 0.0,
                                                                 "wall": 0.0, "fallback": 0.0}}
           for a in arms}
    t_e = t_b = 0.0
    pool = 0
    for q in evalq:
        N.decompose_search([q])   # untimed: builds the candidate space once
        for m in arms.values():
            m.learned_search(q, K=1024, fallback=True)
        full, dt = timed(lambda: N.decompose_search([q], full=True)[0])
        t_e += dt
        exact, dt = timed(lambda: N.decompose_search([q])[0])
        t_b += dt
        assert exact["index"] == full["index"]
        want = (full["primary_bytes"], full["secondary_bytes"])
        for a, m in arms.items():
            A = acc[a]
            got, dt = timed(lambda: m.learned_search(q, K=1024, fallback=True))
            A["s"] += dt
            ok = (got["primary_bytes"], got["secondary_bytes"]) == want
            A["zero_regret"] += ok
            A["fallbacks"] += got["fallback"]
            A["n_exact"] += got["n_exact"]
            rule = N.CERTIFIED[got["certified"]] if not got["fallback"] else "fallback"
            A["accepted"][rule] = A["accepted"].get(rule, 0) + 1
            R = A["regret_by_rule"].setdefault(rule, {"queries": 0, "zero_regret": 0})
            R["queries"] += 1
            R["zero_regret"] += ok
            for k in A["phase"]:
                A["phase"][k] += got["ms"][k] / n_eval
            raw = m.learned_search(q, K=1024, fallback=False)
            A["zero_regret_top_k_only"] += (raw["primary_bytes"], raw["secondary_bytes"]) == want
            pool = max(pool, raw["n_scored"])
    model.close()
    untrained.close()
    out = {"metric": "pruned vs exhaustive time-to-optimum", "value": t_e / acc["trained"]["s"],
           "unit": "x (speed-up)", "ms_learned_mean": 1e3 * acc["trained"]["s"] / n_eval,
           "ms_exhaustive_mean": 1e3 * t_e / n_eval, "ms_primary_bound_mean": 1e3 * t_b / n_eval,
           "vs_primary_bound": t_b / acc["trained"]["s"], "eval_queries": n_eval, "K": 1024,
           "train_labels": n_train * per_query, "train_epochs": epochs, "train_seconds": t_train,
           "train_final_loss": loss, "calibration_queries": n_cal, "calibration_seconds": t_cal,
           "models_trained": len(bounds), "calibration_bounds": bounds, "margin_bound": bound,
           "largest_scored_pool": pool}
    for a in arms:
        A = acc[a]
        out[a] = {"ms_mean": 1e3 * A["s"] / n_eval, "vs_primary_bound": t_b / A["s"],
                  "zero_regret": A["zero_regret"] / n_eval,
                  "zero_regret_top_k_only": A["zero_regret_top_k_only"] / n_eval,
                  "fallbacks": A["fallbacks"], "exact_evaluations_mean": A["n_exact"] / n_eval,
                  "accepted_by": A["accepted"], "zero_regret_by_rule": A["regret_by_rule"],
                  "phase_ms_mean": A["phase"]}
    return out


# multiply-adds per training sample: forward 64*256 + 2*256*256, the three
# weight gradients as many again, and the two hidden-layer input gradients
# 2*256*256 (the output layer's 256 + 256 are left out)
TRAIN_FLOP_PER_SAMPLE = 2 * (147456 + 147456 + 131072)


def sustained_bf16_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["bf16_tflops_sustained"]), "measured"
    except (OSError, KeyError, ValueError):
        return 1700.0, "fallback"


SCORE_FLOP_PER_CANDIDATE = 2 * (64 * 256 + 2 * 256 * 256 + 256)


def burst_bf16_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["bf16_tflops"]), "measured"
    except (OSError, KeyError, ValueError):
        return 1900.0, "fallback"


def extra_scorer(N, W, torch, dev, reps=7):
    """The learned scorer's layer kernel (k_mlp_img: three tcgen05 layers and
    the output dot product) timed alone with CUDA events around one full
    launch of 2^19 candidates (the first run of scoring every candidate of the
    P = 3600 search query, by a briefly trained model): TFLOP/s and the
    fraction of the measured BF16 burst peak (the kernel is timed alone)."""
    q = _search_query_3600()
    m = N.MLP(seed=11)
    m.train_search(W.search_training_queries(16), samples_per_query=1024, epochs=1, batch=1024, lr=1e-3, seed=3)
    nf, nc = N.search_space(q["machine"][0] * q["machine"][1], q["machine"][1], q["max_depth"])
    scores = torch.empty(nf * nc, dtype=torch.float32, device=dev)
    m.scores(q, scores)   # warm: the candidate space and the scoring buffers
    torch.cuda.synchronize()
    ms = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()   # once here, so that torch reads them after the library records them again
        b.record()
        torch.cuda.synchronize()
        N.set_layer_timer(a, b)
        m.scores(q, scores)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    m.close()
    med = sorted(ms)[len(ms) // 2]
    cands = 1 << 19
    tflops = cands * SCORE_FLOP_PER_CANDIDATE / (med * 1e-3) / 1e12
    peak, src = burst_bf16_peak()
    return {"metric": "layer kernel TFLOP/s (BF16)", "value": tflops, "unit": "TFLOP/s", "frac_of_peak": tflops / peak,
            "peak_tflops": peak, "peak_source": f"{src} bf16_tflops (burst)", "ms_per_launch": med,
            "ms_launches": ms, "candidates_per_launch": cands, "flop_per_candidate": SCORE_FLOP_PER_CANDIDATE,
            "workload": "every candidate of the P = 3600 matmul search query (256 x 1024 x 4096 tiles on 450 x 8), "
                        "first run of 2^19"}


def extra_train(N, torch, dev, batch=4096, steps=300, warmup=10):
    """Training steps of the learned cost model (forward, backward and Adam
    on one batch of 4096 samples, every product on the tcgen05 GEMM):
    samples/s, achieved TFLOP/s of the products and the fraction of the
    sustained BF16 peak."""
    g = torch.Generator(device="cpu").manual_seed(5)
    X = torch.randn(batch, 64, generator=g).to(torch.bfloat16).to(dev)
    t = torch.randn(batch, generator=g).to(dev)
    m = N.MLP(seed=5)
    for _ in range(warmup):
        m.train_step(X, t, lr=1e-4)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        m.train_step(X, t, lr=1e-4)
    e1.record()
    torch.cuda.synchronize()
    m.close()
    ms = e0.elapsed_time(e1) / steps
    tflops = TRAIN_FLOP_PER_SAMPLE * batch / (ms / 1e3) / 1e12
    peak, kind = sustained_bf16_peak()
    return {"metric": "training samples/s", "value": batch / (ms / 1e3), "unit": "samples/s", "batch": batch,
            "ms_per_step": ms, "tflops": tflops, "peak_tflops": peak, "peak_source": f"{kind} bf16_tflops_sustained",
            "frac_of_peak": tflops / peak, "flop_per_sample": TRAIN_FLOP_PER_SAMPLE,
            "note": "each step synchronises once (it returns the loss), and its GEMMs are 128-row tiles "
                    "of 4096 x 256 x {64, 256} and 256 x {64, 256} x 4096 products"}


def extra_volume_study(N, W, torch, dev):
    """Decompose vs the greedy grid of Algorithm A1 on the paper's 180-config
    stencil grid: exact halo volume (width 1, 8-byte elements) of the block
    mapping on each grid, computed by the engine."""
    cfgs = W.stencil_study_configs()
    total = torch.empty(1, dtype=torch.int64, device=dev)
    rows = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for c in cfgs:
        G = c["gpus"]
        g = N.greedy_grid(G, 2)
        vols = []
        for chain in ([("merge", 0, 1), ("split", 0, g[0])], [("merge", 0, 1), ("decompose", 0, c["L"])]):
            N.halo_volume(c["L"], c["machine"], chain, ("block",), (1, 1), (8, 8), total=total)
            vols.append(int(total.item()))
        rows.append((c, vols[0], vols[1]))
    secs = time.perf_counter() - t0

    def gmean_improvement(sel):
        ratios = [vg / vd for c, vg, vd in rows if sel(c) and vd > 0]
        gm = math.exp(sum(math.log(v) for v in ratios) / len(ratios))
        return 1.0 - 1.0 / gm

    by = lambda key, vals: {str(v): round(100 * gmean_improvement(lambda c, v=v: c[key] == v), 2) for v in vals}
    return {"metric": "halo volume reduction of decompose over the greedy grid",
            "unit": "% (geometric mean over configurations)",
            "value": round(100 * gmean_improvement(lambda c: True), 2),
            "configs": len(rows), "max_pct": round(100 * max(1 - vd / vg for _, vg, vd in rows), 2),
            "by_aspect_ratio": by("ratio", W.STUDY_RATIOS), "by_points_per_node": by("area", W.STUDY_AREAS),
            "by_gpus": by("gpus", W.STUDY_GPUS), "seconds": secs}


def extra_hier_search(N, W, torch):
    """Two-level (node grid x GPU grid) search on the large launch's task
    space and machine, both variants: exact inter-node and inter-processor
    element halo volumes of every candidate on the GPU."""
    L, machine = W.large_config("block")["L"], W.large_config("block")["machine"]
    out = {}
    for variant in ("block", "cyclic"):
        N.hier_search(L, machine, variant, (1, 1, 1), (8, 8, 8))   # warm
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = N.hier_search(L, machine, variant, (1, 1, 1), (8, 8, 8))
        dt = time.perf_counter() - t0
        out[variant] = {"ms": 1e3 * dt, "candidates": r["n_candidates"], "a": r["a"], "b": r["b"],
                        "inter_node_bytes": r["primary"], "inter_proc_bytes": r["secondary"]}
    cands = sum(v["candidates"] for v in out.values())
    secs = sum(v["ms"] for v in out.values()) / 1e3
    return {"metric": "two-level candidates/s", "value": cands / secs, "unit": "candidates/s",
            "workload": "1024x1024x512 on 64 x 8, node grid x GPU grid, width-1 element halo", **out}


def extra_applications(N, W, torch, dev, reps=5):
    """ids + histogram + halo of launches shaped like the paper's
    applications (Circuit, PENNANT, stencil, Cannon, SUMMA, PUMMA,
    Johnson/COSMA) on 64 x 8: points/s and the id stream's GB/s."""
    out = []
    for w in W.application_shapes():
        npts = math.prod(w["L"])
        P = w["machine"][0] * w["machine"][1]
        ids = torch.empty(npts, dtype=torch.int32, device=dev)
        hist = torch.empty(P, dtype=torch.int64, device=dev)
        total = torch.empty(1, dtype=torch.int64, device=dev)
        recv = torch.empty(P, dtype=torch.int64, device=dev)

        def once():
            N.map_launch(w["L"], w["machine"], w["chain"], w["dist"], ids=ids, hist=hist, face_bytes=w["face"],
                         total=total, recv=recv)

        for _ in range(2):
            once()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            once()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        out.append({"workload": w["name"], "L": list(w["L"]), "points": npts, "ms": ms,
                    "points_per_s": npts / (ms / 1e3), "ids_gbs": 4 * npts / (ms / 1e3) / 1e9})
        del ids, hist, total, recv
    torch.cuda.empty_cache()
    pts = sum(o["points"] for o in out)
    secs = sum(o["ms"] for o in out) / 1e3
    return {"metric": "points mapped/s", "value": pts / secs, "unit": "points/s",
            "note": "ids + histogram + halo per launch, one call each", "launches": out}


def max_over_ranks(value: float, dist, device) -> float:
    """The largest value of all ranks (the job is as slow as its slowest
    rank); the value itself without a process group."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_reference(args, rank, world):
    """The CPU oracle timed on the host cores: each step maps a bounded sample
    of the large launch (sized so that the whole run ends in a few minutes)."""
    if rank != 0:
        return
    steps = max(1, args.steps)
    per_step = max(1 << 14, min(1 << 24, (1 << 29) // (steps + max(args.warmup, 0))))
    times = []
    info = None
    for _ in range(max(args.warmup, 0)):
        cpu_baseline(max(per_step // 8, 4096), single_core=False)
    for _ in range(steps):
        info = cpu_baseline(per_step, single_core=False)
        times.append(info["seconds"])
    total_s = sum(times)
    value = per_step * steps / total_s
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_s / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic",
            "config": {"workload": "large launch: 1024x1024x512 points on 64 nodes x 8 procs, seeded random "
                                   "split/merge/swap chain depth 4 (CPU oracle, bounded sample per step)",
                       "sample_points_per_step": per_step},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": info["cores"], "kind": "oracle",
                             "sample": info["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def profile_case_ids(N, torch):
    """256 x 1024 x 512 points (512 MiB of ids, larger than L2), the block
    variant's chain, mapped four times."""
    cfg = W.large_config("block")
    L = (256, 1024, 512)
    chain = N.chain_from_draws(*cfg["machine"], cfg["draws"])
    ids = torch.empty(math.prod(L), dtype=torch.int32, device="cuda")
    for _ in range(4):
        N.map_points(L, cfg["machine"], chain, cfg["dist"], ids=ids)


def _search_query_3600():
    return [q for q in W.search_queries(16) if q["machine"][0] * q["machine"][1] == 3600][0]


def profile_case_search(N, torch):
    """The exhaustive search (every candidate's secondary scanned) of the first
    P = 3600 query of the search workload, twice."""
    q = _search_query_3600()
    for _ in range(2):
        N.decompose_search([q], full=True)


def profile_case_score(N, torch):
    """Fused scoring of every candidate of the same query (3.8 M candidates)
    by a briefly trained model, twice."""
    m = N.MLP(seed=11)
    m.train_search(W.search_training_queries(16), samples_per_query=1024, epochs=1, batch=1024, lr=1e-3, seed=3)
    q = _search_query_3600()
    for _ in range(2):
        m.learned_search(q, K=1024, fallback=False, score_all=True)
    m.close()


def profile_case_score_features(N, torch):
    """The same scoring, then the feature generator alone over every
    candidate (k_features_idx writes the 64 BF16 features of each), to split
    the scorer's time between features and the layers."""
    m = N.MLP(seed=11)
    q = _search_query_3600()
    n = 3787020
    scores = torch.empty(n, dtype=torch.float32, device="cuda")
    feats = torch.empty((n + 127) // 128 * 128, 64, dtype=torch.bfloat16, device="cuda")
    for _ in range(2):
        assert m.scores(q, scores, feats) == n
    m.close()


def profile_case_batched(N, torch):
    """200 queries of the batched workload's recipe with at most 2^22 points
    each (about 7e7 points, 270 MB of ids) in one graph replay, three times."""
    qs = W.batched_queries(200, max_points=1 << 22)
    b = N.Batch([(q["L"], q["machine"], N.chain_from_draws(*q["machine"], q["draws"]), q["dist"], q["face"])
                 for q in qs])
    info = b.info()
    ids = torch.empty(int(info["total_ids"]), dtype=torch.int32, device="cuda")
    hist = torch.empty(int(info["total_procs"]), dtype=torch.int64, device="cuda")
    for _ in range(3):
        b.run(ids=ids, hist=hist)
    torch.cuda.synchronize()
    b.close()


def profile_case_train(N, torch):
    """Training steps of the cost model on one batch of 4096 samples, five
    times (every product through k_gemm_tn)."""
    g = torch.Generator(device="cpu").manual_seed(5)
    X = torch.randn(4096, 64, generator=g).to(torch.bfloat16).cuda()
    t = torch.randn(4096, generator=g).cuda()
    m = N.MLP(seed=5)
    for _ in range(5):
        m.train_step(X, t, lr=1e-4)
    m.close()


def profile_case_learned(N, torch):
    """A briefly trained and calibrated model, then the learned search
    (exact costs of the top 1024, no fallback) on six held-out queries,
    twice each (the first builds each candidate space)."""
    m = N.MLP(seed=11)
    m.train_search(W.search_training_queries(64), samples_per_query=2048, epochs=2, batch=4096, lr=2e-3, seed=3)
    m.calibrate(W.search_training_queries(16, first_index=40000))
    for q in W.search_queries(6, first_index=9000):
        N.decompose_search([q])
        for _ in range(2):
            m.learned_search(q, K=1024, fallback=False)
    m.close()


PROFILE_CASES = {"ids-small": profile_case_ids, "search": profile_case_search, "score": profile_case_score,
                 "train-step": profile_case_train, "learned": profile_case_learned,
                 "score-features": profile_case_score_features, "batched": profile_case_batched}


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if world > 1 and rank != 0:
            return
        run_reference(args, rank, world)
        return

    import torch
    from paper_2507_17087_gb300 import build as B
    from paper_2507_17087_gb300 import native as N

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (the engine has no CPU fallback)")
    B.build()
    torch.cuda.set_device(local)
    if args.profile_case:
        PROFILE_CASES[args.profile_case](N, torch)
        torch.cuda.synchronize()
        print("ok", args.profile_case, flush=True)
        return
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    dev = torch.device("cuda", local)
    cfgs = launches()
    chains = [N.chain_from_draws(*c["machine"], c["draws"]) for c in cfgs]
    L = cfgs[0]["L"]
    P = cfgs[0]["machine"][0] * cfgs[0]["machine"][1]
    npts = math.prod(L)
    ids = torch.empty(npts, dtype=torch.int32, device=dev)
    hist = torch.empty(P, dtype=torch.int64, device=dev)
    total = torch.empty(1, dtype=torch.int64, device=dev)
    recv = torch.empty(P, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(timers=None):
        for v, (cfg, chain) in enumerate(zip(cfgs, chains)):
            if timers is not None:
                N.set_kernel_timer(*timers[v])
            N.map_launch(cfg["L"], cfg["machine"], chain, cfg["dist"], ids=ids, hist=hist, face_bytes=cfg["face"],
                         total=total, recv=recv, stream=stream)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()

    # per-launch CUDA events around the id writer (the dominant kernel)
    kev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            for _ in VARIANTS] for _ in range(args.steps)]
    for pairs in kev:
        for a, b in pairs:
            a.record(stream)
            b.record(stream)
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = N.kernel_launches()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for s in range(args.steps):
        step(kev[s])
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    gpu_launches = N.kernel_launches() - launches0
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    kms = [a.elapsed_time(b) for pairs in kev for a, b in pairs]
    k_avg_ms = sum(kms) / len(kms)
    ms = max_over_ranks(ms, dist, dev)
    points = 3 * npts * args.steps * world
    value = points / (ms / 1e3)

    # ---------------------------------------------------------------- e2e
    # the same step through the public API with host buffers: the ids, the
    # histogram, the halo total and the received bytes come back to pinned host
    # memory inside the timed region; the launch description goes down as
    # kernel parameters.
    h_ids = torch.empty(npts, dtype=torch.int32).pin_memory()
    h_hist = torch.empty(P, dtype=torch.int64).pin_memory()
    h_total = torch.empty(1, dtype=torch.int64).pin_memory()
    h_recv = torch.empty(P, dtype=torch.int64).pin_memory()
    launches_before = N.kernel_launches()

    def e2e_step():
        for cfg, chain in zip(cfgs, chains):
            N.map_launch(cfg["L"], cfg["machine"], chain, cfg["dist"], ids=h_ids, hist=h_hist, face_bytes=cfg["face"],
                         total=h_total, recv=h_recv, stream=stream)

    e2e_step()
    per_step_launches = N.kernel_launches() - launches_before
    # three trials of the same steps, the median reported (a host-link hiccup
    # during one trial does not set the number)
    trials = []
    for _ in range(3):
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            e2e_step()
        trials.append(max_over_ranks(time.perf_counter() - t0, dist, dev))
    e2e_s = sorted(trials)[1]
    e2e_value = 3 * npts * args.e2e_steps * world / e2e_s
    d2h = 3 * (npts * 4 + P * 8 + 8 + P * 8)
    h2d = per_step_launches * N.descriptor_bytes()

    if rank == 0:
        peak, peak_kind = peaks()
        algo_bytes = 4 * npts
        achieved = algo_bytes / (k_avg_ms / 1e3) / 1e9
        traffic = K_IDS_TRAFFIC_BYTES
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": "large launch: 1024x1024x512 points on 64 nodes x 8 procs, seeded random "
                                   "split/merge/swap chain depth 4, block + cyclic + block-cyclic(4), "
                                   "7-point halo 8 B",
                       "points_per_step": 3 * npts, "parallelism": f"replicas x{world}",
                       "l2": "outputs larger than L2 (2 GiB of ids per launch)"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "traffic_source": "ncu capture of one full-size k_ids launch (dram read + write "
                                           "bytes), taken separately, not in this run",
                         "kernel": "k_ids (id writer)", "peak_source": f"{peak_kind} hbm_gbs",
                         "kernel_avg_ms": k_avg_ms, "algorithmic_bytes_per_launch": algo_bytes,
                         "note": "k_ids only writes, and hbm_gbs is a read + write copy: a write-only "
                                 "2 GiB fill moves 7.2-7.75 TB/s on the same GPUs"},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "timing": "median of 3 trials of %d steps (host wall clock)" % args.e2e_steps,
                    "trial_values": [3 * npts * args.e2e_steps * world / t for t in trials]},
            "gpu_launches": gpu_launches,
            "clocks": clocks,
        }
        if not args.no_extras:
            for key, fn in (("search", lambda: extra_search(N, W, torch)),
                            ("batched", lambda: extra_batched(N, W, torch, dev)),
                            ("learned", lambda: extra_learned(N, W, torch)),
                            ("train", lambda: extra_train(N, torch, dev)),
                            ("scorer", lambda: extra_scorer(N, W, torch, dev)),
                            ("volume_study", lambda: extra_volume_study(N, W, torch, dev)),
                            ("hier_search", lambda: extra_hier_search(N, W, torch)),
                            ("applications", lambda: extra_applications(N, W, torch, dev))):
                try:
                    line[key] = fn()
                except Exception as exc:  # noqa: BLE001 - an extra must not lose the main line
                    line[key] = {"error": f"{type(exc).__name__}: {exc}"}
        if not args.no_cpu_baseline and world == 1:
            try:
                cb = cpu_baseline(args.cpu_sample)
                cb.pop("seconds", None)
                line["cpu_baseline"] = cb
            except Exception as exc:  # noqa: BLE001
                line["cpu_baseline"] = {"error": str(exc)}
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
