#!/usr/bin/env python3
"""Throughput benchmark of the ACE hot path (insert + score points/s).

Workload: the KDD-shaped configuration — n = 500,000 binary32 rows, d = 41, a 23-cluster
Gaussian mixture min-max normalised to [0,1] plus 1% uniform anomalies, K = 15, L = 50,
alpha = 1 (synthetic stand-in for KDD-Cup99 HTTP).  One step = one ace_insert_score call on
one batch: hash every point (Eq. 1-2), insert it (Algorithm 1 counting phase), then gather
every point's score against the updated arrays and flag it (query phase + §5.3 rule).
Inputs are resident in HBM before the timed region; steps rotate over three distinct
batches (3 x 82 MB > 129 MB L2), so no step reads its input from L2.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision auto|fp32|bf16]
  python bench.py --impl reference ...   # the CPU oracle on a bounded sample (baseline arm)

Prints one JSON line (rank 0).
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
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "insert+score points/s per config vs plain FP32 GPU path; % roofline; p99 latency"
UNIT = "points/s"
WORKLOAD = "kdd-shaped n=500000 d=41 K=15 L=50 alpha=1 (23-cluster mixture, 1% uniform anomalies)"
N_POINTS, D, KH, LT, ALPHA = 500_000, 41, 15, 50, 1.0
# The high-dimensional workload (--workload highdim; profiling and per-config runs): bfloat16
# points drawn on the device, d = 1024, K = 16, L = 64.
HIGHDIM = {"n": 1_000_000, "d": 1024, "K": 16, "L": 64,
           "name": "high-dimensional n=1000000 d=1024 K=16 L=64 bf16 (64 clusters on the unit sphere, 0.5% anomalies)"}
FP32_ALU_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12  # SMs x FP32 lanes x 2 x max SM clock

REF_BUDGET_S = 90.0  # timed CPU work of one --impl reference run

PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
PROFILE_EVERY = 8  # one timed step in PROFILE_EVERY has its dominant kernel bracketed by events
TRAFFIC_PATH = os.path.join(ROOT, "profiles", "traffic.json")


def _peaks():
    try:
        with open(PEAKS_PATH) as f:
            p = json.load(f)
        return {"hbm_gbs": p["hbm_gbs"], "bf16_tflops": p["bf16_tflops"],
                "bf16_tflops_sustained": p.get("bf16_tflops_sustained"), "src": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "src": "fallback"}


# sources that determine each timed kernel's code (its traffic figure is void once one changes)
KERNEL_SOURCES = {
    "hash_tc": ("hash_tc.cu", "tc_ptx.cuh", "tc_plan.h", "guard.cuh", "ace_internal.h", "exact_div.h"),
    "hash_simt": ("hash_simt.cu", "guard.cuh", "ace_internal.h", "exact_div.h", "score_block.cuh", "flag_wait.cuh"),
    "hash_gemm": ("hash_gemm.cu", "gemm_plan.h", "tc_ptx.cuh", "guard.cuh", "ace_internal.h", "exact_div.h"),
    "hash_gemm_fp8": ("hash_gemm.cu", "gemm_plan.h", "tc_ptx.cuh", "guard.cuh", "ace_internal.h", "exact_div.h"),
    "hash_fwht": ("hash_fwht.cu", "fwht_plan.h", "guard.cuh", "ace_internal.h", "exact_div.h", "f32x2.cuh",
                  "fwht_exact.cuh"),
}


def _src_sha(kernel_key: str) -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel_key]:
        with open(os.path.join(ROOT, "paper_1706_06664_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _traffic(kernel_key: str, units: int):
    """DRAM bytes per launch from the committed ncu summary, if the kernel is unchanged."""
    try:
        with open(TRAFFIC_PATH) as f:
            t = json.load(f)[kernel_key]
    except Exception:
        return None
    if t.get("src_sha") != _src_sha(kernel_key):
        return None
    return t["bytes_per_point"] * units


class Clocks:
    """Samples nvidia-smi clocks and throttle reasons in the background."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
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
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx = float(parts[2])
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, 0, None
    import torch.distributed as dist
    rank, local = int(os.environ["RANK"]), int(os.environ.get("LOCAL_RANK", "0"))
    import torch
    if torch.cuda.is_available():
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        dist.init_process_group("gloo")
    return rank, ws, local, dist


def _max_over_ranks(x: float, dist, device):
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _batches(rank: int, n: int):
    from paper_1706_06664_gb300 import workloads
    return [workloads.kdd(seed=2 + 1000 * rank + 10 * b, n=n)["X"] for b in range(3)]


def _device_batches(rank: int, n: int, count: int = 2):
    """The high-dimensional batches, drawn on the device (2 x 2 GB at n = 1,000,000)."""
    from paper_1706_06664_gb300 import workloads
    return [workloads.highdim_device(seed=3 + 1000 * rank + 10 * b, n=n)[0] for b in range(count)]


def cpu_baseline(X: np.ndarray, detector_seed: int, budget_s: float = 12.0) -> dict:
    """The CPU oracle as it stands, on a bounded prefix of one batch (insert + score)."""
    import oracle
    ref = oracle.Detector(D, KH, LT, seed=detector_seed)
    probe = min(2000, X.shape[0])
    t0 = time.perf_counter()
    ref.insert_score(X[:probe], ALPHA)
    per_pt = (time.perf_counter() - t0) / probe
    m = int(min(X.shape[0], max(probe, budget_s / max(per_pt, 1e-9))))
    ref = oracle.Detector(D, KH, LT, seed=detector_seed)
    t0 = time.perf_counter()
    ref.insert_score(X[:m], ALPHA)
    dt = time.perf_counter() - t0
    return {"value": m / dt, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"insert_score of the first {m} points of one {X.shape[0]}-point batch "
                      f"({dt:.1f} s, binary64 C oracle, OpenMP over points)"}


def _config_cases():
    """The small and KDD-shaped configs at full size (host batches) and the high-dimensional one
    at its full size, n = 1,000,000, drawn on the device (its host generator takes minutes at
    that size); the CPU oracle times the high-dimensional config on a host draw of the same
    recipe (its rate per point does not depend on n)."""
    from paper_1706_06664_gb300 import workloads
    Xd, _ = workloads.highdim_device(seed=3, n=1_000_000)
    c3 = {"X_dev": Xd, "d": 1024, "K": 16, "L": 64, "dtype": "bf16", "w_bf16_variant": True,
          "X": workloads.highdim(seed=3, n=20_000)["X"]}
    return [("small", workloads.small(seed=1)), ("kdd-shaped", workloads.kdd(seed=2)),
            ("high-dimensional", c3)]


def oracle_per_config(cases, budget_s: float = 1.5) -> dict:
    """The CPU oracle's insert+score rate per config, on all host cores and on one core:
    insert_score on a fresh detector over a prefix of the config's (host) batch sized to about
    budget_s seconds (a 200-point probe sets the size)."""
    import oracle
    out = {}
    all_cores = oracle.num_threads()
    try:
        for name, w in cases:
            X = w["X"]
            res = {}
            for cores in (all_cores, 1):
                oracle.set_num_threads(cores)
                probe = min(200, X.shape[0])
                t0 = time.perf_counter()
                oracle.Detector(w["d"], w["K"], w["L"], seed=11).insert_score(X[:probe], ALPHA)
                per_pt = (time.perf_counter() - t0) / probe
                m = int(min(X.shape[0], max(probe, budget_s / max(per_pt, 1e-9))))
                ref = oracle.Detector(w["d"], w["K"], w["L"], seed=11)
                t0 = time.perf_counter()
                ref.insert_score(X[:m], ALPHA)
                dt = time.perf_counter() - t0
                res[f"{cores}_cores"] = {"points_per_s": m / dt, "sample_points": m}
            out[name] = res
    finally:
        oracle.set_num_threads(all_cores)
    return out


def count_phases(n: int, K: int, L: int, phases_ms: dict) -> dict:
    """The counting and query phases against library baselines of the same work, probed in the
    same run: the insert's n L count increments against uniformly random 32-bit atomic
    additions straight into the L2-resident L 2^K counts (torch index_add_: the L2-atomic way
    of counting, at its no-contention rate), and the score's n L gathers against uniformly
    random 4-byte loads from that array (torch take, 64-bit indices, one output per load).
    ratio > 1: the library kernels' way is slower (the insert uses privatised shared-memory
    histograms instead of L2 atomics).  CUDA events, median of 5 after 2 warm-up runs."""
    import torch
    dev = torch.device("cuda")
    m = n * L
    counts = torch.zeros(L << K, dtype=torch.int32, device=dev)
    g = torch.Generator(device=dev)
    g.manual_seed(5)
    idx = torch.randint(0, L << K, (m,), device=dev, generator=g)
    ones = torch.ones(m, dtype=torch.int32, device=dev)

    def timed(fn):
        ts = []
        for r in range(7):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            if r >= 2:
                ts.append(e0.elapsed_time(e1) / 1e3)
        return statistics.median(ts)

    t_atom = timed(lambda: counts.index_add_(0, idx, ones))
    t_take = timed(lambda: torch.take(counts, idx))
    out = {"increments_or_gathers_per_step": m,
           "probe_note": "library baselines probed in this run on uniformly random addresses of an "
                         f"L2-resident array of {L << K} counts ({(L << K) * 4 / 1e6:.1f} MB)"}
    for name, key, tp, pk in (("insert", "insert", t_atom, "l2_atomic_probe_per_s"),
                              ("score_gather", "score", t_take, "library_gather_probe_per_s")):
        if key in phases_ms and phases_ms[key] > 0:
            ach = m / (phases_ms[key] / 1e3)
            out[name] = {"achieved_per_s": ach, pk: m / tp, "ratio": ach / (m / tp)}
    del counts, idx, ones
    return out


def _step_roofline(n, d, K, L, x_bytes, ms, peaks):
    """The whole call against its roofline, the slower of its bytes and its flop:
    t_roof = max((X + W bytes) / HBM, projection flop / bf16 peak), with the measured peaks;
    frac = t_roof / measured time."""
    flop = 2.0 * n * d * K * L
    byt = n * d * x_bytes + d * K * L * 4
    t_roof = max(byt / (peaks["hbm_gbs"] * 1e9), flop / (peaks["bf16_tflops"] * 1e12))
    return {"t_roof_ms": t_roof * 1e3, "frac": t_roof / (ms / 1e3),
            "bound": "tensor" if flop / (peaks["bf16_tflops"] * 1e12) >= byt / (peaks["hbm_gbs"] * 1e9) else "hbm",
            "peaks": f"{peaks['hbm_gbs']:.0f} GB/s, {peaks['bf16_tflops']:.0f} TFLOP/s bf16 ({peaks['src']})"}


PRIVACY_SIGMA = 1.0


def per_config(cases) -> dict:
    """insert+score points/s per config on each engine it runs on, against the plain binary32
    (FP32) engine: CUDA events on the launching stream around each call, median of 10 calls
    after 3 warm-up calls on one detector per engine, the batch resident in HBM; the hash
    kernel's own time from the library's timing hook (its roofline fraction in algorithmic
    flop against the measured bf16 peak), and the whole call against its roofline
    (_step_roofline).  The batched and streaming configs have sections of their own."""
    import torch
    from paper_1706_06664_gb300 import ace
    stream = torch.cuda.current_stream()
    peaks = _peaks()
    out = {}
    for name, w in cases:
        if "X_dev" in w:
            Xd = w["X_dev"]
        else:
            X = w["X"]
            Xd = torch.from_numpy(X.view(np.int16) if X.dtype == np.uint16 else X).cuda()
        n = Xd.shape[0]
        xb = 2 if w.get("dtype") == "bf16" else 4
        flop = 2.0 * n * w["d"] * w["K"] * w["L"]
        res = {"n": n, "d": w["d"], "K": w["K"], "L": w["L"], "x_dtype": "bf16" if xb == 2 else "f32"}
        variants = [("fp32", ace.ACE_PROJ_FP32, {}), ("bf16", ace.ACE_PROJ_BF16, {})]
        if w.get("w_bf16_variant"):
            variants.append(("bf16_w_bf16", ace.ACE_PROJ_BF16, {"w_bf16": True}))
            variants.append(("fp8_w_bf16", ace.ACE_PROJ_FP8, {"w_bf16": True}))
        # the structured +-1 projection (a different hash family: other ids, its own roofline)
        variants.append(("fwht_hadamard", ace.ACE_PROJ_FWHT, {"w_hadamard": True}))
        if n <= 100_000:  # launch-bound batches: repeated calls replayed as a captured CUDA graph
            variants.append(("fp32_graph", ace.ACE_PROJ_FP32, {"graph": True}))
            variants.append(("bf16_graph", ace.ACE_PROJ_BF16, {"graph": True}))
        # §4.5 privacy noise before the sign (sigma = 1): the cost of drawing and adding it
        variants.append(("fp32_privacy", ace.ACE_PROJ_FP32, {"privacy": PRIVACY_SIGMA}))
        variants.append(("fwht_hadamard_privacy", ace.ACE_PROJ_FWHT, {"w_hadamard": True, "privacy": PRIVACY_SIGMA}))
        for prec, want, kw in variants:
            kw = dict(kw)
            sigma = kw.pop("privacy", 0.0)
            graph = kw.pop("graph", False)
            try:
                det = ace.Detector(w["d"], w["K"], w["L"], seed=11, precision=prec.split("_")[0], **kw)
                if sigma:
                    det.set_privacy(sigma, 12)
            except ace.AceError as e:
                if e.code == ace.ACE_ERR_UNSUPPORTED:
                    res[prec] = "engine not available for this shape"
                    continue
                raise
            reps = 13 if not (prec == "fp32" and n * w["d"] * w["K"] * w["L"] > 1e11) else 5
            times = []
            if graph:
                # replay needs the same arguments every call (fixed outputs) on a stream of its
                # own; the timing hook would turn it off, so no phases are read
                det.set_graph(True)
                gs = torch.cuda.Stream()
                outs = (torch.empty(n, dtype=torch.float64, device=Xd.device),
                        torch.empty(n, dtype=torch.int32, device=Xd.device),
                        torch.empty(n, dtype=torch.uint8, device=Xd.device))
                reps = 23
                for r in range(reps):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(gs)
                    det.insert_score(Xd, ALPHA, *outs, stream=gs)
                    e1.record(gs)
                    torch.cuda.synchronize()
                    if r >= 3:
                        times.append(e0.elapsed_time(e1) / 1e3)
            else:
                for r in range(reps):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    if r == 3:
                        det.profile_read()
                        det.profile(True)
                    e0.record(stream)
                    det.insert_score(Xd, ALPHA, stream=stream)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    if r >= 3:
                        times.append(e0.elapsed_time(e1) / 1e3)
            det.profile(False)
            prof = det.profile_read()
            st = det.stats()
            used = st["precision"]
            det.close()
            if used != want:
                res[prec] = "engine not used for this shape"
                continue
            t = statistics.median(times)
            phases = {k: v["ms"] / v["timed"] for k, v in prof.items() if v["timed"]}
            entry = {"points_per_s": n / t, "ms": t * 1e3, "projection_tflops": flop / t / 1e12,
                     "tc_products": st["tc_products"],
                     "phases_ms": phases, "rechecks_per_point": st["rechecks"] / (n * reps),
                     "deferred_per_point": st["deferred"] / (n * reps),
                     "step_roofline": _step_roofline(n, w["d"], w["K"], w["L"], xb, t * 1e3, peaks)}
            if sigma:
                entry["privacy_sigma"] = sigma
            if "hash" in phases:
                th = phases["hash"] / 1e3
                if prec.startswith("bf16"):
                    entry["hash_roofline"] = {"bound": "tensor", "achieved": flop / th / 1e12,
                                              "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
                                              "frac": flop / th / 1e12 / peaks["bf16_tflops"],
                                              "peak_src": f"bf16 burst, {peaks['src']}"}
                elif prec.startswith("fwht"):
                    # HBM-bound: X read once, ids written once (2 or 4 bytes per table)
                    byts = n * (w["d"] * xb + w["L"] * (2 if w["K"] <= 16 else 4))
                    entry["hash_roofline"] = {"bound": "hbm", "achieved": byts / th / 1e9, "peak": peaks["hbm_gbs"],
                                              "unit": "GB/s", "frac": byts / th / 1e9 / peaks["hbm_gbs"],
                                              "peak_src": f"HBM copy, {peaks['src']}"}
                elif prec.startswith("fp8"):
                    pk = 2.0 * peaks["bf16_tflops"]
                    entry["hash_roofline"] = {"bound": "tensor", "achieved": flop / th / 1e12, "peak": pk,
                                              "unit": "TFLOP/s", "frac": flop / th / 1e12 / pk,
                                              "peak_src": f"fp8 dense = 2 x bf16 burst ({peaks['src']}; nominal ratio)"}
                else:
                    entry["hash_roofline"] = {"bound": "alu", "achieved": flop / th / 1e12, "peak": FP32_ALU_PEAK_TFLOPS,
                                              "unit": "TFLOP/s", "frac": flop / th / 1e12 / FP32_ALU_PEAK_TFLOPS,
                                              "peak_src": "FP32 FMA: 152 SMs x 128 lanes x 2 flop x 2070 MHz (derived)"}
            res[prec] = entry
        for v in ("bf16", "bf16_w_bf16", "fp8_w_bf16", "fwht_hadamard", "fp32_privacy", "fp32_graph", "bf16_graph"):
            if isinstance(res.get(v), dict) and isinstance(res.get("fp32"), dict):
                res[f"{v}_vs_fp32"] = res[v]["points_per_s"] / res["fp32"]["points_per_s"]
        if isinstance(res.get("fwht_hadamard_privacy"), dict) and isinstance(res.get("fwht_hadamard"), dict):
            res["fwht_hadamard_privacy_vs_fwht_hadamard"] = (res["fwht_hadamard_privacy"]["points_per_s"] /
                                                             res["fwht_hadamard"]["points_per_s"])
        out[name] = res
        del Xd
    return out


def run_reference(args):
    if int(os.environ.get("RANK", "0")) != 0:
        return 0  # the CPU oracle runs on rank 0 only
    import oracle
    X = _batches(0, N_POINTS)[0]
    # Size each step so the timed steps take about REF_BUDGET_S in all, whatever --steps is.
    probe = 2000
    t0 = time.perf_counter()
    oracle.Detector(D, KH, LT, seed=7).insert_score(X[:probe], ALPHA)
    per_pt = (time.perf_counter() - t0) / probe
    sample = int(max(1000, min(args.ref_sample, args.ref_budget / max(1, args.steps) / max(per_pt, 1e-9))))
    for _ in range(args.warmup):
        oracle.Detector(D, KH, LT, seed=7).insert_score(X[:max(1, sample // 10)], ALPHA)
    times = []
    for s in range(args.steps):
        ref = oracle.Detector(D, KH, LT, seed=7)
        off = (s * sample) % max(1, X.shape[0] - sample)
        t0 = time.perf_counter()
        ref.insert_score(X[off:off + sample], ALPHA)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = sample * args.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "sample_points_per_step": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": f"{sample} points of the batch per step (insert_score)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _e2e(args, det, host_batches, stream, dist, dev, n, ws):
    import torch
    det.reset()
    pin_x = [torch.from_numpy(b).pin_memory() for b in host_batches]
    hx = [p.numpy() for p in pin_x]
    o_sc = torch.empty(n, dtype=torch.float64).pin_memory().numpy()
    o_su = torch.empty(n, dtype=torch.int32).pin_memory().numpy().view(np.uint32)
    o_fl = torch.empty(n, dtype=torch.uint8).pin_memory().numpy()
    # the streaming host entry: each step enqueues its batch (copy in, insert + score, copy
    # out); the copy of one step overlaps the computation of the previous one
    for i in range(2):
        det.insert_score_host_async(hx[i % len(hx)], ALPHA, o_sc, o_su, o_fl, stream=stream)
    det.host_wait()
    det.reset()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    for i in range(args.steps):
        det.insert_score_host_async(hx[i % len(hx)], ALPHA, o_sc, o_su, o_fl, stream=stream)
    det.host_wait()
    e2e_s = _max_over_ranks(time.perf_counter() - t0, dist, dev)
    # the host link's own rate for the same bytes: one plain pinned copy of a batch, best of 10
    dst = torch.empty(pin_x[0].numel(), dtype=pin_x[0].dtype, device=dev)
    with torch.cuda.stream(stream):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        link = []
        for _ in range(10):
            ev0.record(stream)
            dst.view(-1).copy_(pin_x[0].view(-1), non_blocking=True)
            ev1.record(stream)
            ev1.synchronize()
            link.append(ev0.elapsed_time(ev1))
    link_gbs = pin_x[0].nbytes / (min(link) / 1e3) / 1e9
    x_gbs = pin_x[0].nbytes * args.steps / e2e_s / 1e9
    return {"value": n * args.steps * ws / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(hx[0].nbytes),
            "d2h_bytes_per_step": int(o_sc.nbytes + o_su.nbytes + o_fl.nbytes),
            "x_gbs": x_gbs, "host_link_gbs": link_gbs, "of_link": x_gbs / link_gbs,
            "link_note": "x_gbs: X bytes moved per second end to end (per rank); host_link_gbs: one plain "
                         "pinned host-to-device copy of a batch on the same stream, best of 10"}


def serving(seed: int = 31, window_points: int = 1 << 20, n_windows: int = 4, n_det: int = 64,
            n_req: int = 3000) -> dict:
    """Streaming-serving shape: 64 detectors (d=128, K=15, L=50), request sizes log-uniform
    in [1, 8192], inserts and scores 50/50 on random detectors, points from four windows of
    1,048,576 consecutive points of the 100,000,000-point drifting stream, at its start, a
    quarter, half and three quarters of the way (so requests see means from across the
    drift).  Capacity from the best of three closed-loop bursts (a single burst varied by up to
    1.5x from run to run); then Poisson arrivals at 0.5x, 0.8x and 1.0x that rate, paced by a
    spin that yields the CPU; latency = submission to completion (outputs in host memory).  Run
    in a process of its own (serving_isolated) so that no state of the other measurements
    carries over."""
    import torch
    from paper_1706_06664_gb300 import ace, workloads
    d, K, L = 128, 15, 50
    total = 100_000_000
    dets = [ace.Detector(d, K, L, seed=1000 + i) for i in range(n_det)]
    starts = [w * (total // n_windows) for w in range(n_windows)]
    pool = torch.from_numpy(np.concatenate([workloads.stream_chunk(seed, st, window_points, total=total, d=d)
                                            for st in starts])).pin_memory().numpy()
    pool_points = pool.shape[0]
    rng = np.random.default_rng(seed)
    srv = ace.Server(dets, mem_budget_bytes=1 << 30)

    def workload(count, salt):
        sizes = workloads.request_sizes(seed + salt, count)
        # a random window, then consecutive requests walk through it
        win = rng.integers(0, n_windows, size=count)
        offs = win * window_points + (np.concatenate([[0], np.cumsum(sizes)[:-1]]) % (window_points - 8192))
        ops = rng.integers(0, 2, size=count)  # 0 insert, 1 score
        dsel = rng.integers(0, n_det, size=count)
        out = torch.empty(int(sizes.sum()) * 13 + 64 * (count + 1), dtype=torch.uint8).pin_memory().numpy()
        return sizes, offs, ops, dsel, out

    def submit_all(sizes, offs, ops, dsel, out, arrivals=None):
        # the requests' arrays are cut before the clock starts: the timed loop only submits
        reqs, pos = [], 0
        for k in range(len(sizes)):
            n = int(sizes[k])
            X = pool[offs[k]:offs[k] + n]
            if ops[k] == 0:
                reqs.append((int(dsel[k]), ace.OP_INSERT, X, 1.0, None, None, None))
            else:
                sc = out[pos:pos + 8 * n].view(np.float64)
                su = out[pos + 8 * n:pos + 12 * n].view(np.uint32)
                fl = out[pos + 12 * n:pos + 13 * n]
                pos = (pos + 13 * n + 63) // 64 * 64
                reqs.append((int(dsel[k]), ace.OP_SCORE, X, 1.0, sc, su, fl))
        tickets = []
        submit = srv.submit
        t0 = time.perf_counter()
        for k, r in enumerate(reqs):
            if arrivals is not None:
                while time.perf_counter() - t0 < arrivals[k]:
                    os.sched_yield()
            tickets.append(submit(*r))
        t_sub = time.perf_counter() - t0
        lat = np.array([srv.wait(t) for t in tickets])
        return lat, time.perf_counter() - t0, t_sub

    # every detector starts with 8192 inserted points
    for i in range(n_det):
        srv.wait(srv.submit(i, ace.OP_INSERT, pool[i * 8192:(i + 1) * 8192]))
    w = workload(n_req, 1)
    submit_all(*w)  # warm-up (buffers grow to their final sizes)
    best = None
    for salt in (2, 22, 42):
        w = workload(n_req, salt)
        lat, el, t_sub = submit_all(*w)
        if best is None or float(w[0].sum()) / el > best[1]:
            best = (n_req / el, float(w[0].sum()) / el, lat, el, t_sub)
    cap_req, cap_pts, lat, cap_el, cap_sub = best
    res = {"workload": f"drifting stream d={d} K={K} L={L} ({total} points; requests drawn from {n_windows} "
                       f"windows of {window_points} points at {starts}), {n_det} detectors, requests log-uniform "
                       f"1-8192, 50/50 insert/score, {n_req} requests per run",
           "capacity": {"points_per_s": cap_pts, "requests_per_s": cap_req,
                        "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                        # the Python client's own submission time: when it is most of the burst, the
                        # client, not the server, set the rate (no queue formed)
                        "submit_s": cap_sub, "elapsed_s": cap_el, "client_bound": bool(cap_sub > 0.8 * cap_el)}}
    for f in (0.5, 0.8, 1.0):
        w = workload(n_req, 3 + int(f * 10))
        arrivals = np.cumsum(rng.exponential(1.0 / (f * cap_req), size=n_req))
        lat, el, _ = submit_all(*w, arrivals=arrivals)
        res[f"load_{f}"] = {"points_per_s": float(w[0].sum()) / el, "p50_ms": float(np.percentile(lat, 50) * 1e3),
                            "p99_ms": float(np.percentile(lat, 99) * 1e3)}
    res["scheduler"] = srv.info()  # threads; requests admitted inside another insert's launch set
    srv.close()
    for dd in dets:
        dd.close()
    return res


def serving_isolated() -> dict:
    """serving() in a fresh interpreter (its own CUDA context)."""
    code = "import json, bench; print(json.dumps(bench.serving()))"
    out = subprocess.run([sys.executable, "-c", code], cwd=os.path.dirname(os.path.abspath(__file__)),
                         capture_output=True, text=True, check=True)
    return json.loads(out.stdout.strip().splitlines()[-1])


def projection_errors() -> dict:
    """Per config and engine: max and mean of |estimate - binary64| / (||x|| ||w_c||) over a
    sample (estimates from ace_project, binary64 from the oracle), and rechecks per point of an
    insert_score of the same sample."""
    import torch
    import oracle
    from paper_1706_06664_gb300 import ace, workloads
    cases = [("small", workloads.small(seed=1, n=4000), ("fp32", "bf16")),
             ("kdd-shaped", workloads.kdd(seed=2, n=20000), ("fp32", "bf16")),
             ("high-dimensional (d=1024, bf16 input)", workloads.highdim(seed=3, n=1000),
              ("fp32", "bf16", "bf16_w_bf16", "fp8_w_bf16"))]
    out = {}
    for name, w, precs in cases:
        X = w["X"]
        Xd = torch.from_numpy(X.view(np.int16) if X.dtype == np.uint16 else X).cuda()
        Xf = workloads.bf16_bits_to_f32(X) if X.dtype == np.uint16 else X
        res = {}
        for prec in precs:
            det = ace.Detector(w["d"], w["K"], w["L"], seed=5, precision=prec.split("_")[0],
                               w_bf16=prec.endswith("w_bf16"))
            est = det.project(Xd).cpu().numpy().astype(np.float64)
            W = det.projection()
            s64 = oracle.project(X, W)
            rel = np.abs(est - s64) / (np.linalg.norm(Xf.astype(np.float64), axis=1)[:, None] *
                                       np.linalg.norm(W.astype(np.float64), axis=0)[None, :])
            det.insert_score(Xd, ALPHA)
            torch.cuda.synchronize()
            res[prec] = {"max": float(rel.max()), "mean": float(rel.mean()),
                         "rechecks_per_point": det.stats()["rechecks"] / X.shape[0]}
            det.close()
        out[f"{name}: n={X.shape[0]} d={w['d']} K={w['K']} L={w['L']}"] = res
    return out


def estimator_accuracy(seed: int = 12, m: int = 50, Ls=(10, 25, 50, 100, 200)) -> dict:
    """Estimator-accuracy workload (§4.2; stand-ins for the paper's datasets, which are not
    available): for 50 queries drawn from each dataset, the exact S(q, D) of Eq. 3 on the GPU
    (ace_exact_score, binary64), ACE's estimate at L arrays and RSE with L samples (20 draws);
    mean square error against L.  Also the exact-score kernel's rate: 4 d binary64 flop per
    (query, point) pair (dot product and the point's squared norm), against the nominal 1.25
    TFLOP/s binary64 rate of the part."""
    import torch
    from paper_1706_06664_gb300 import accuracy, ace, workloads
    sets = [("small-shaped (n=10000, d=32)", workloads.small(seed=1)["X"], 15),
            ("kdd-shaped (n=100000, d=41)", workloads.kdd(seed=2, n=100_000)["X"], 15),
            ("high-dimensional (n=100000, d=1024 bf16)", workloads.highdim(seed=3, n=100_000)["X"], 15)]
    out = {}
    for name, X, K in sets:
        Xd = torch.from_numpy(X.view(np.int16) if X.dtype == np.uint16 else X).cuda()
        rng = np.random.default_rng(seed)
        Q = Xd[torch.from_numpy(rng.choice(X.shape[0], size=m, replace=False)).cuda()]
        res = accuracy.estimator_mse(Xd, Q, K, Ls, seed=seed, rse_draws=20)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ace.exact_score(Q, Xd, K)
        e0.record()
        ace.exact_score(Q, Xd, K)
        e1.record()
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        pairs = m * X.shape[0]
        out[name] = {"K": K, "queries": m, "mean_S": float(np.mean(res["S"])),
                     "mse": {str(L): {"ace": v["ace_mse"], "rse": v["rse_mse"]} for L, v in res["L"].items()},
                     "exact_score": {"pairs_per_s": pairs / t, "ms": t * 1e3,
                                     "fp64_tflops": 4.0 * X.shape[1] * pairs / t / 1e12,
                                     "frac_of_nominal_fp64": 4.0 * X.shape[1] * pairs / t / 1.25e12}}
    return out


def batched(n_det: int = 2048, seed: int = 4) -> dict:
    """Batched-detectors shape: 2048 detectors, d log-uniform in [16, 512], n log-uniform in
    [100, 100000], K=12, L=32, Gaussian-mixture points (8 clusters N(m_c, I), m_c ~ N(0, 4I),
    1% shifted by +4 in 3 dimensions) drawn on the device from a seeded generator.  One
    ace_batch_insert_score call against the same work as one ace_insert_score per detector."""
    import torch
    from paper_1706_06664_gb300 import ace, workloads
    specs = workloads.batched_specs(seed=seed, n_det=n_det)
    K, L = 12, 32
    g = torch.Generator(device="cuda").manual_seed(seed)
    Xs = []
    for (d, n, sd) in specs:
        means = 2.0 * torch.randn(8, d, device="cuda", generator=g)
        which = torch.randint(0, 8, (n,), device="cuda", generator=g)
        X = means[which] + torch.randn(n, d, device="cuda", generator=g)
        k = max(1, n // 100)
        X[torch.randint(0, n, (k,), device="cuda", generator=g)[:, None],
          torch.randint(0, d, (min(3, d),), device="cuda", generator=g)[None, :]] += 4.0
        Xs.append(X.contiguous())
    points = int(sum(n for _, n, _ in specs))
    dets = [ace.Detector(d, K, L, seed=sd, precision="fp32") for (d, _, sd) in specs]
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ace.batch_insert_score(dets, Xs)  # warm-up: scratch grows to size
    torch.cuda.synchronize()
    ev[0].record(stream)
    ace.batch_insert_score(dets, Xs)
    ev[1].record(stream)
    for det, X in zip(dets, Xs):
        det.insert_score(X, ALPHA)
    ev[2].record(stream)
    torch.cuda.synchronize()
    t_b, t_l = ev[0].elapsed_time(ev[1]) / 1e3, ev[1].elapsed_time(ev[2]) / 1e3
    for det in dets:
        det.close()
    # the same batch with W regenerated from each detector's seed inside the kernel
    # (ACE_W_COUNTER: no row-major W is stored or read)
    dets = [ace.Detector(d, K, L, seed=sd, precision="fp32", w_counter=True) for (d, _, sd) in specs]
    ace.batch_insert_score(dets, Xs)
    torch.cuda.synchronize()
    ev[0].record(stream)
    ace.batch_insert_score(dets, Xs)
    ev[1].record(stream)
    torch.cuda.synchronize()
    t_c = ev[0].elapsed_time(ev[1]) / 1e3
    for det in dets:
        det.close()
    w_bytes = sum(d * K * L * 4 for (d, _, _) in specs)
    return {"workload": f"{n_det} detectors, d log-uniform 16-512, n log-uniform 100-100000, K={K} L={L}, "
                        f"{points} points, binary32 engine",
            "points_per_s": points / t_b, "ms": t_b * 1e3,
            "one_call_per_detector_points_per_s": points / t_l, "one_call_per_detector_ms": t_l * 1e3,
            "counter_w": {"points_per_s": points / t_c, "ms": t_c * 1e3, "w_bytes_not_stored": w_bytes,
                          "note": "ACE_W_COUNTER detectors: W tiles regenerated from the seed in the kernel "
                                  "(integer-only generator; a different W, so other ids)"}}


def run_ours(args):
    import torch
    from paper_1706_06664_gb300 import ace

    rank, ws, local, dist = _dist()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (the library has no CPU path)")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    n = args.n
    if args.workload == "highdim":
        X = _device_batches(rank, n)
        host_batches = None  # drawn on the device; the e2e pass copies them to pinned host memory
    else:
        host_batches = _batches(rank, n)
        X = [torch.from_numpy(b).to(dev) for b in host_batches]
    seed = 1234 + rank
    det = ace.Detector(D, KH, LT, seed=seed, precision=args.precision, w_bf16=args.w_bf16, w_hadamard=args.w_hadamard)
    stream = torch.cuda.current_stream(dev)
    sc = torch.empty(n, dtype=torch.float64, device=dev)
    su = torch.empty(n, dtype=torch.int32, device=dev)
    fl = torch.empty(n, dtype=torch.uint8, device=dev)

    def step(i):
        det.insert_score(X[i % len(X)], ALPHA, scores=sc, sums=su, flags=fl, stream=stream)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    # Per-phase breakdown from a short pass with every kernel bracketed by events (those events
    # cost about 9 % of a step); the timed steps then bracket only the dominant kernel, whose
    # live duration the roofline needs.
    det.profile_read()
    det.profile(True)
    pre = min(50, max(1, args.steps))
    for i in range(pre):
        step(i)
    torch.cuda.synchronize()
    det.profile(False)
    pre_prof = {k: v for k, v in det.profile_read().items() if v["timed"]}
    top = max(pre_prof, key=lambda k: pre_prof[k]["ms"])
    det.reset()
    det.profile_read()
    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.3)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(args.steps):
        sampled = i % PROFILE_EVERY == 0
        if sampled:
            det.profile(True, phases=[top])
        step(i)
        if sampled:
            det.profile(False)
    e1.record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    ck = clocks.stop()
    det.profile(False)
    prof = det.profile_read()
    st = det.stats()
    ms = e0.elapsed_time(e1)
    ms_max = _max_over_ranks(ms, dist, dev)
    value = n * args.steps * ws / (ms_max / 1e3)

    # ---- end to end through the host-buffer entry point --------------------------------
    e2e = None
    if args.e2e:
        if host_batches is None:
            host_batches = [x.cpu().numpy().view(np.uint16) for x in X]
        e2e = _e2e(args, det, host_batches, stream, dist, dev, n, ws)

    # ---- roofline of the dominant kernel --------------------------------------------
    peaks = _peaks()
    ph = {k: v for k, v in prof.items() if v["timed"]}
    per_launch_ms = {k: v["ms"] / v["timed"] for k, v in ph.items()}
    precision = st["precision"]
    flops = 2.0 * n * D * KH * LT
    if top == "hash":
        t = per_launch_ms["hash"] / 1e3
        if precision == ace.ACE_PROJ_BF16:
            kkey = "hash_tc" if D <= 64 else "hash_gemm"
            roof = {"bound": "tensor", "achieved": flops / t / 1e12, "peak": peaks["bf16_tflops"],
                    "unit": "TFLOP/s", "peak_src": f"bf16 burst, {peaks['src']}"}
        elif precision == ace.ACE_PROJ_FWHT:
            kkey = "hash_fwht"
            byts = n * (D * (2 if args.workload == "highdim" else 4) + LT * (2 if KH <= 16 else 4))
            roof = {"bound": "hbm", "achieved": byts / t / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "peak_src": f"HBM copy, {peaks['src']}"}
        elif precision == ace.ACE_PROJ_FP8:
            kkey = "hash_gemm_fp8"
            roof = {"bound": "tensor", "achieved": flops / t / 1e12, "peak": 2.0 * peaks["bf16_tflops"],
                    "unit": "TFLOP/s",
                    "peak_src": f"fp8 dense = 2 x bf16 burst ({peaks['src']}; nominal 4.5 / 2.25 PFLOP/s ratio)"}
        else:
            kkey = "hash_simt"
            roof = {"bound": "alu", "achieved": flops / t / 1e12, "peak": FP32_ALU_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "peak_src": "FP32 FMA: 152 SMs x 128 lanes x 2 flop x 2070 MHz (derived)"}
        roof["traffic"] = _traffic(kkey, n)
        roof["kernel"] = kkey
    else:
        t = per_launch_ms[top] / 1e3
        algo = n * LT * (2 + 4) + n * 4  # ids read + one 4-byte count per gather + sums write
        roof = {"bound": "hbm", "achieved": algo / t / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "traffic": None, "kernel": top}
    roof["frac"] = roof["achieved"] / roof["peak"]

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {ace.ACE_PROJ_BF16: "bf16", ace.ACE_PROJ_FP8: "e4m3"}.get(precision, "f32"), "data": "synthetic",
        "config": {"workload": WORKLOAD, "precision": ["fp32", "bf16", "fp8", "fwht"][precision] if precision in (0, 1, 2, 3) else precision,
                   "l2": ("inputs rotate over 2 resident batches (2 x 2 GB > 129 MB L2)" if args.workload == "highdim"
                          else "inputs rotate over 3 resident batches (246 MB > 129 MB L2)"),
                   "w": "structured +-1 (Hadamard rows, random signs)" if args.w_hadamard else ("bfloat16-valued" if args.w_bf16 else "binary32"),
                   "parallelism": f"replicas x{ws} (independent detectors, no collective)"},
        "roofline": roof,
        "step_roofline": _step_roofline(n, D, KH, LT, 2 if args.workload == "highdim" else 4, ms_max / args.steps,
                                        peaks),
        "phases_ms_per_step": {k: v["ms"] / pre for k, v in pre_prof.items()},
        "phases_note": f"from {pre} steps with every kernel bracketed by CUDA events, before the timed "
                       f"steps; in the timed steps only '{top}' (the roofline's kernel) is bracketed, "
                       f"on every {PROFILE_EVERY}th step",
        "rechecks_per_point": st["rechecks"] / max(1, n * args.steps),
        "e2e": e2e,
        "gpu_launches": int(sum(v["launches"] for v in prof.values())),
        "clocks": ck,
    }
    # The sections below add context to the line; a failure in one is reported in its place
    # rather than losing the measurement above.
    def section(fn, *a):
        try:
            return fn(*a)
        except Exception as e:  # noqa: BLE001 - reported in the JSON line
            return {"error": f"{type(e).__name__}: {e}"[:300]}

    if rank == 0 and ws == 1:
        line["count_phases"] = section(count_phases, n, KH, LT, line["phases_ms_per_step"])
    cases = None
    if rank == 0 and ws == 1 and (args.per_config or args.cpu_baseline):
        cases = section(_config_cases)
        if isinstance(cases, dict):  # the generators failed
            line["per_config"], cases = cases, None
    if rank == 0 and ws == 1 and args.per_config and cases is not None:
        line["per_config"] = section(per_config, cases)
    if rank == 0 and args.cpu_baseline and host_batches is not None and args.workload == "kdd":
        line["cpu_baseline"] = section(cpu_baseline, host_batches[0], seed)
        if cases is not None and "error" not in line["cpu_baseline"]:
            line["cpu_baseline"]["per_config"] = section(oracle_per_config, cases)
    if rank == 0 and ws == 1 and args.serving:
        line["serving"] = section(serving_isolated)
    if rank == 0 and ws == 1 and args.batched:
        line["batched"] = section(batched)
    if rank == 0 and ws == 1 and args.proj_error:
        line["projection_error"] = section(projection_errors)
    if rank == 0 and ws == 1 and args.accuracy:
        line["estimator_accuracy"] = section(estimator_accuracy)
    if rank == 0:
        print(json.dumps(line), flush=True)
    det.close()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="auto", choices=["auto", "fp32", "bf16", "fp8", "fwht"])
    ap.add_argument("--n", type=int, default=None, help="points per batch (profiling runs only)")
    ap.add_argument("--workload", default="kdd", choices=["kdd", "highdim"],
                    help="kdd: the headline KDD-shaped workload; highdim: d = 1024 bfloat16 (profiling runs)")
    ap.add_argument("--w-bf16", dest="w_bf16", action="store_true", help="draw W in bfloat16 (ace_create_ex)")
    ap.add_argument("--w-hadamard", dest="w_hadamard", action="store_true",
                    help="structured +-1 W (ACE_W_HADAMARD); with --precision fwht or auto, the transform engine")
    ap.add_argument("--ref-sample", type=int, default=100_000, help="points per reference step")
    ap.add_argument("--ref-budget", type=float, default=REF_BUDGET_S, help="seconds of timed reference work")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-e2e", dest="e2e", action="store_false")
    ap.add_argument("--no-serving", dest="serving", action="store_false")
    ap.add_argument("--no-batched", dest="batched", action="store_false")
    ap.add_argument("--no-projection-error", dest="proj_error", action="store_false")
    ap.add_argument("--no-per-config", dest="per_config", action="store_false")
    ap.add_argument("--no-accuracy", dest="accuracy", action="store_false")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)  # at least 3 untimed warm-up steps
    global D, KH, LT, WORKLOAD
    if args.workload == "highdim":
        D, KH, LT, WORKLOAD = HIGHDIM["d"], HIGHDIM["K"], HIGHDIM["L"], HIGHDIM["name"]
        if args.n is None:
            args.n = HIGHDIM["n"]
    if args.n is None:
        args.n = N_POINTS
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
