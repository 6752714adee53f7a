"""Benchmark: SBV log-likelihood evaluations per second on one GB300.

Workload (default): sine10d -- n = 1,000,000 points uniform on [0,1]^10, y from
the sine-sum family, 20,000 K-means blocks (~50 points), m = 120 neighbours,
Matern-5/2, one theta per evaluation (the shape of the paper's Sec. 8
performance study: d = 10 on [0,1]^10).  Blocking and kNN run once, untimed
(reported separately); a step is one full log-likelihood evaluation: gather,
covariance, factorisation, refinement, block terms and the deterministic sum.

The headline is the mixed path (SBV_PREC_MIXED); the FP64 path and the
tensor-core split-BF16 variant are timed beside it on the same structure,
with |l_path - l_fp64| / n.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  `--impl reference` times the FP64 CPU oracle on host
cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import re
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

METRIC = "SBV loglik evals/s & TFLOP/s on 1 GB300, mixed vs FP64 at |dl|/n <= 1e-6"
UNIT = "evals/s"
L2_BYTES = 129 * 1024 * 1024
# FP32 CUDA-core peak from unit counts and clock: 152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# FP64 peak: 1.25 TFLOP/s nominal for GB300 (a DFMA probe measured 1.19-1.20)
FP64_PEAK_TFLOPS = 1.25
# the sources of the mixed block kernel (the recorded traffic is valid for these)
KERNEL_SRC = [os.path.join(ROOT, "paper_2504_12004_gb300", "csrc", f)
              for f in ("loglik_mixed.cu", "mixed.cuh", "dfloat.cuh", "block_common.cuh")]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "loglik_mixed_sine10d_traffic.txt")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="sine10d")
    p.add_argument("--n", type=int, default=None, help="shrink the workload (profiling runs)")
    p.add_argument("--bc", type=int, default=None, help="blocks of the shrunk workload")
    p.add_argument("--precision", default="mixed", choices=["mixed", "mixed_bf16", "fp64"])
    p.add_argument("--kmeans-iters", type=int, default=10)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-side-paths", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--launch", default="graph", choices=["graph", "direct"],
                   help="time graph replays (default) or direct sbv_loglik calls")
    p.add_argument("--no-autotune", action="store_true")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running.

    nvidia-smi stalls the device for a few hundred ms while it starts, so the
    sampler is started before the warm-up and only samples whose timestamps
    fall inside the timed window (set by window()) are summarised."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t0 = self.t1 = None

    def window(self, t0: float, t1: float):
        self.t0, self.t1 = t0, t1

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for t, l in self.lines:
            # a line is read shortly after its sample; keep the timed window (+ one period)
            if self.t0 is not None and not (self.t0 <= t <= self.t1 + 0.25):
                continue
            parts = [x.strip() for x in l.split(",")]
            if len(parts) < 10:
                continue
            try:
                sm.append(float(parts[2]))
                mx.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[6:10]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- helpers
def make_workload(name: str, n=None, bc=None):
    from synth.inputs import workload
    w = workload(name, n=n, bc=bc)
    if w["y"] is None:
        raise SystemExit(f"workload {name} needs a GP draw; use a sine-sum workload for the bench")
    return w


def algorithmic_flops(ptr: np.ndarray, cnt: np.ndarray) -> float:
    """sum_i N_i^3/3 + N_i^2 (Cholesky of the joint matrix plus the bordered solve)."""
    N = np.diff(ptr).astype(np.float64) + cnt.astype(np.float64)
    return float(np.sum(N ** 3 / 3.0 + N ** 2))


def kernel_pairs(ptr: np.ndarray, cnt: np.ndarray) -> float:
    N = np.diff(ptr).astype(np.float64) + cnt.astype(np.float64)
    return float(np.sum(N * (N + 1) / 2))


def source_hash(paths) -> str:
    """sha256 (16 hex) of the kernel sources with comments and whitespace removed,
    so that a recorded capture stays valid across comment-only edits."""
    h = hashlib.sha256()
    for path in paths:
        with open(path, encoding="utf-8") as f:
            text = f.read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


def recorded_traffic(workload: str):
    """DRAM bytes per launch of the mixed kernel recorded from ncu, if the kernel source is unchanged."""
    try:
        kv = {}
        with open(TRAFFIC_FILE) as f:
            for line in f:
                if ":" in line:
                    k, v = line.split(":", 1)
                    kv[k.strip()] = v.strip()
        if kv.get("workload") == workload and kv.get("source_sha256_16") == source_hash(KERNEL_SRC):
            return float(kv["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


# ----------------------------------------------------------------------------- CPU baseline
CPU_SNIPPET = r"""
import json, sys, time
import numpy as np
sys.path.insert(0, {root!r})
from synth.inputs import workload
from oracle import sbv
w = workload({name!r})
n, bc, m = w["n"], w["bc"], w["m"]
bs = n // bc
# the oracle's per-block arithmetic depends only on the block's size and neighbour
# count: a smaller point set with the same bs and m gives full-size blocks to time
nb = {nblocks}
nsub = min(n, nb * bs)
X = w["X"][:nsub]; y = w["y"][:nsub]
b = sbv.blocking(X, w["beta_scale"], nsub // bs, 0, 5)
nbr, cnt = sbv.knn(b["Z"], b["blk"], b["rank"], b["centres"], m)
rows = np.nonzero(cnt == min(m, int(cnt.max())))[0]
th = w["theta"][0]
done = 0
t0 = time.perf_counter()
while time.perf_counter() - t0 < {seconds}:
    sbv.loglik_terms(X, y, b["ptr"], b["pts"], nbr, cnt, th, w["nu2"], blocks=rows)
    done += rows.size
dt = time.perf_counter() - t0
print(json.dumps(dict(seconds=dt, blocks=int(done), distinct=int(rows.size), bc=bc, bs=bs, m=m)))
"""


def cpu_baseline(name: str, seconds: float, nblocks: int = 400):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    code = CPU_SNIPPET.format(root=ROOT, name=name, nblocks=nblocks, seconds=seconds)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                       timeout=1200)
    if r.returncode != 0:
        return {"error": r.stderr[-400:]}
    res = json.loads(r.stdout.strip().splitlines()[-1])
    per_block = res["seconds"] / res["blocks"]
    evals_per_s = 1.0 / (per_block * res["bc"])
    return {"value": evals_per_s, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{res['blocks']} block terms ({res['distinct']} distinct full-size blocks, "
                      f"bs~{res['bs']}, m={res['m']}) of the {name} workload shape in "
                      f"{res['seconds']:.1f} s of single-thread FP64 oracle time, extrapolated "
                      f"linearly to bc={res['bc']}"}


# ----------------------------------------------------------------------------- reference arm
def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from synth.inputs import WORKLOADS
    w = WORKLOADS[args.workload]
    per_step = []
    secs = max(2.0, min(args.cpu_seconds, 120.0 / max(1, args.steps + args.warmup)))
    for i in range(args.warmup + args.steps):
        cb = cpu_baseline(args.workload, secs)
        if "error" in cb:
            print(json.dumps({"impl": "reference", "unavailable": cb["error"][-200:]}))
            return
        if i >= args.warmup:
            per_step.append(cb)
    v = statistics.median([c["value"] for c in per_step])
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 / v,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "n": w["n"], "d": w["d"], "bc": w["bc"],
                   "m": w["m"], "nu": w["nu2"] / 2, "theta_per_eval": 1},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": per_step[-1]["sample"]},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ----------------------------------------------------------------------------- our arm
def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    import torch.distributed as dist
    from paper_2504_12004_gb300 import build, Context

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    build.build()
    ctx = Context(local)
    dev = torch.device("cuda", local)

    # ---------------- inputs (synthetic, seeded) and one-time structure
    w = make_workload(args.workload, args.n, args.bc)
    X_h, y_h, beta, th = w["X"], w["y"], w["beta_scale"], w["theta"]
    X = torch.from_numpy(X_h).to(dev)
    y = torch.from_numpy(y_h).to(dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b = ctx.sbv_blocking(X, beta, w["bc"], args.kmeans_iters, 1234)
    torch.cuda.synchronize()
    t_block = time.perf_counter() - t0
    t0 = time.perf_counter()
    nbr, cnt = ctx.sbv_knn(X, beta, b["ptr"], b["pts"], b["rank"], b["centres"], w["m"])
    torch.cuda.synchronize()
    t_knn = time.perf_counter() - t0
    ptr, pts = b["ptr"], b["pts"]
    bc = b["bc_eff"]
    nbr = nbr.contiguous()
    ptr_h, cnt_h = ptr.cpu().numpy(), cnt.cpu().numpy()
    flops = algorithmic_flops(ptr_h, cnt_h)
    pairs = kernel_pairs(ptr_h, cnt_h)
    Nsz = np.diff(ptr_h) + cnt_h

    nmax = ctx.max_block_size(ptr, cnt)

    # launch shape from the autotuner, then one evaluation captured as a CUDA
    # graph (counter reset, persistent block kernel, fixed-order reduction)
    # and replayed with the parameter row as its only input
    tuned = None
    if not args.no_autotune:
        tuned = ctx.sbv_autotune(X, y, ptr, pts, nbr, cnt, th, nu2=w["nu2"],
                                 precision=args.precision, nmax=nmax)
    graph = None
    if args.launch == "graph":
        graph = ctx.sbv_loglik_graph_create(X, y, ptr, pts, nbr, cnt, B=1, nu2=w["nu2"],
                                            precision=args.precision, nmax=nmax)

    def evaluate(precision):
        if graph is not None and precision == args.precision:
            return graph.launch(th)
        return ctx.sbv_loglik(X, y, ptr, pts, nbr, cnt, th, nu2=w["nu2"], precision=precision,
                              nmax=nmax)

    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    flush.fill_(0.0)                 # first use of the fill costs ~0.25 s once: keep it untimed
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()

    def timed(prec, steps, warmup, clk=None):
        for _ in range(warmup):
            evaluate(prec)
        torch.cuda.synchronize()
        if clk is not None:
            time.sleep(1.5)              # let the sampler finish starting up before timing
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t_wall0 = time.time()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        start = torch.cuda.Event(enable_timing=True)
        end = torch.cuda.Event(enable_timing=True)
        start.record(stream)
        out = None
        for i in range(steps):
            flush.fill_(float(i))        # evict L2 between steps (inputs would otherwise stay resident)
            ev[i][0].record(stream)
            out = evaluate(prec)
            ev[i][1].record(stream)
        end.record(stream)
        torch.cuda.synchronize()
        if clk is not None:
            clk.window(t_wall0, time.time())
        if world > 1:
            dist.barrier()
        total_ms = start.elapsed_time(end)
        per_call = [a.elapsed_time(c) for a, c in ev]
        return total_ms, per_call, out

    precision = args.precision
    with ClockSampler(local) as clk:
        total_ms, per_call, ll = timed(precision, args.steps, args.warmup, clk)
    clocks = clk.summary()
    if world > 1:
        tt = torch.tensor([total_ms], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        total_ms = float(tt.item())
    ll_v = float(ll[0].item())
    value = world * args.steps / (total_ms / 1000.0)
    call_ms = statistics.median(per_call)

    # side paths on the same structure and theta
    paths = {precision: {"evals_per_s": value, "ms_per_call": call_ms, "ll": ll_v}}
    if not args.no_side_paths:
        for prec in ("fp64", "mixed", "mixed_bf16"):
            if prec in paths:
                continue
            k = max(3, args.steps // 4)
            t_tot, t_calls, t_ll = timed(prec, k, 1)
            paths[prec] = {"evals_per_s": k / (t_tot / 1000.0), "ms_per_call": statistics.median(t_calls),
                           "ll": float(t_ll[0].item())}
    if "fp64" in paths:
        ref = paths["fp64"]["ll"]
        for p in paths.values():
            p["delta_l_per_n_vs_fp64"] = abs(p["ll"] - ref) / w["n"]
        paths["speedup_vs_fp64"] = paths["fp64"]["ms_per_call"] / call_ms
    if not args.no_side_paths:
        # FP64 value and analytic gradient in theta (sbv_loglik_grad), same
        # structure and theta; L2 flushed before every timed call
        try:
            for _ in range(2):
                gl, gg = ctx.sbv_loglik_grad(X, y, ptr, pts, nbr, cnt, th, nu2=w["nu2"], nmax=nmax)
            torch.cuda.synchronize()
            g_ms = []
            for i in range(3):
                flush.fill_(float(i))
                a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a0.record(stream)
                gl, gg = ctx.sbv_loglik_grad(X, y, ptr, pts, nbr, cnt, th, nu2=w["nu2"], nmax=nmax)
                a1.record(stream)
                torch.cuda.synchronize()
                g_ms.append(a0.elapsed_time(a1))
            g_call = statistics.median(g_ms)
            entry = {"evals_per_s": 1000.0 / g_call, "ms_per_call": g_call, "ll": float(gl[0].item()),
                     "gradient_components": int(gg.shape[1])}
            if "fp64" in paths:
                entry["ll_equals_fp64_path"] = entry["ll"] == paths["fp64"]["ll"]
            paths["fp64_value_and_gradient"] = entry
        except Exception as e:  # a side measurement never costs the headline line
            paths["fp64_value_and_gradient"] = {"error": str(e)[:200]}

    # ---------------- end to end: host buffers in, host scalar out, copies timed
    pin = lambda t: t.cpu().pin_memory()
    host = {k: pin(v) for k, v in dict(X=X, y=y, ptr=ptr, pts=pts, nbr=nbr, cnt=cnt).items()}
    dev_bufs = {k: torch.empty_like(v, device=dev) for k, v in host.items()}
    ll_host = torch.empty(1, dtype=torch.float64).pin_memory()
    h2d = sum(v.numel() * v.element_size() for v in host.values())
    for i in range(args.warmup + args.steps):
        if i == args.warmup:
            torch.cuda.synchronize()
            e0 = time.perf_counter()
        for k, v in host.items():
            dev_bufs[k].copy_(v, non_blocking=True)
        o = ctx.sbv_loglik(dev_bufs["X"], dev_bufs["y"], dev_bufs["ptr"], dev_bufs["pts"],
                           dev_bufs["nbr"], dev_bufs["cnt"], th, nu2=w["nu2"], precision=precision,
                           nmax=nmax)
        ll_host.copy_(o, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = time.perf_counter() - e0
    e2e = {"value": world * args.steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
           "d2h_bytes_per_step": 8}

    # ---------------- roofline of the dominant kernel (the block log-likelihood)
    achieved_tflops = flops / (call_ms / 1000.0) / 1e12
    if precision == "fp64":
        roof = {"bound": "alu", "achieved": achieved_tflops, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": achieved_tflops / FP64_PEAK_TFLOPS, "traffic": None,
                "peak_source": "nominal FP64 rate of GB300 (DFMA probe measured 1.19)"}
    else:
        roof = {"bound": "alu", "achieved": achieved_tflops, "peak": FP32_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": achieved_tflops / FP32_PEAK_TFLOPS,
                "traffic": recorded_traffic(args.workload) if precision == "mixed" else None,
                "peak_source": "FP32 CUDA-core rate from 152 SMs x 128 lanes x 2 x 2.07 GHz",
                "note": "achieved counts the Cholesky flops sum N^3/3 + N^2 only; the "
                        "double-float covariance (%.3g kernel evaluations per call) is the "
                        "larger share of the issued instructions" % pairs}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.workload, args.cpu_seconds)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if precision == "fp64" else "f32+df64",
            "data": "synthetic",
            "config": {"workload": args.workload, "n": w["n"], "d": w["d"], "bc": bc, "m": w["m"],
                       "nu": w["nu2"] / 2, "theta_per_eval": 1, "precision": precision,
                       "block_N": {"min": int(Nsz.min()), "p50": float(np.median(Nsz)),
                                   "p99": float(np.percentile(Nsz, 99)), "max": int(Nsz.max())},
                       "l2": "flushed between steps (256 MB write)",
                       "parallelism": "replicas" if world > 1 else "single"},
            "tflops": achieved_tflops,
            "kernel_evals_per_s": pairs / (call_ms / 1000.0),
            "ll": ll_v,
            "paths": paths,
            "preprocess_s": {"blocking": t_block, "knn": t_knn},
            "algorithmic_flops_per_eval": flops,
            # graph replay: block kernel + reduction per step; direct call:
            # also the float-pair split of the points
            "gpu_launches": (2 if graph is not None else 3) * args.steps,
            "launch": {"mode": args.launch,
                       "shape": {"threads": tuned[0], "ctas_per_sm": tuned[1]} if tuned else None},
            "clocks": clocks,
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": e2e,
        }
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
