"""Benchmark: exact bivariate resultants per second on one GB300 (or N, one
process per GPU, independent batches: weak scaling).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload batch|single]
                    [--impl ours|reference] [--no-baseline]

Prints ONE JSON line.  A step is one pass of the whole path (G1 reduce +
evaluate + univariate resultants, G2 interpolation, G3 CRT) over one batch of
synthetic input (default: 512 pairs, per-pair deg_x, deg_y ~ U[8, 40],
bidegree-dense, coefficient bits in {16, 32, 64}).  ``value`` is the batched
throughput with inputs resident on the device; ``per_instance`` times the same
kernels launched one pair at a time (no persistence, no graphs); ``e2e`` goes
through the C ABI with host buffers (upload, run, result copy-back);
``cpu_baseline`` times the CPU oracle on a bounded sample.
"""
import argparse
import hashlib
import json
import multiprocessing as mp
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "resultants/s batched vs per-instance launch, same GB300; % of INT32 IMAD peak"
SM_COUNT = 152
IMAD_PER_SM_CLK = 64  # 32-bit integer multiply-add results per clock per SM
WORKLOADS = {
    "batch": "batched: 512 pairs in one run, per-pair deg_x, deg_y ~ U[8,40] shared by f and g, "
             "bidegree-dense, coefficient bits per pair in {16,32,64}, seed 2",
    "single": "single pair, dense total degree 30, signed 32-bit coefficients, seed 1",
}


def load_pairs(workload, npairs=512):
    from paper_1010_1386_gb300 import inputs
    if workload == "batch":
        return inputs.workload_batch(2, n=512)[:npairs]
    return inputs.workload_single(1)


# ------------------------------------------------------------ CPU oracle leg

def _oracle_point(args):
    f, g, x0 = args
    from oracle import exact
    t = time.perf_counter()
    exact.resultant_y_at(f, g, x0)
    return time.perf_counter() - t


def oracle_sample(workload, npairs, seed, cores):
    """Time the oracle's exact Sylvester determinant at the middle evaluation
    point for ``npairs`` sampled pairs (one process each) and extrapolate to
    its full evaluation-interpolation resultant: (D + 1) determinants per pair
    (interpolation not counted).  Returns (resultants/s over ``cores``
    processes, description)."""
    import random
    from paper_1010_1386_gb300 import inputs, rs
    pairs = load_pairs(workload)
    idx = random.Random(seed).sample(range(len(pairs)), min(npairs, len(pairs)))
    jobs, points = [], []
    for i in idx:
        f, g = pairs[i]
        d = rs.result_bound(f, g)["deg"]
        points.append(d + 1)
        jobs.append((f.to_ints(), g.to_ints(), d // 2))
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(cores, len(jobs))) as pool:
        times = pool.map(_oracle_point, jobs)
    per_pair = statistics.mean(t * n for t, n in zip(times, points))
    value = cores / per_pair
    desc = (f"exact integer Sylvester determinant at x = D/2 for {len(jobs)} random pairs "
            f"(mean {statistics.mean(times):.2f} s each), scaled by D+1 points per pair, "
            f"interpolation not counted; {cores} processes")
    return value, desc


# ----------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device, self.proc, self.lines = device, None, []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for name, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# -------------------------------------------------------------- profiles

def g1_traffic():
    """DRAM bytes per G1 stage from the committed ncu summary, if it was taken
    on the current G1 source; else None."""
    path = os.path.join(ROOT, "profiles", "g1_images_batch512.md")
    src = os.path.join(ROOT, "paper_1010_1386_gb300", "csrc", "kernels_g1.cu")
    try:
        text = open(path).read()
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
    except OSError:
        return None
    m_sha = re.search(r"kernels_g1\.cu sha256:\s*([0-9a-f]{64})", text)
    m_tr = re.search(r"dram bytes per G1 stage:\s*([0-9.eE+]+)", text)
    if not m_sha or not m_tr or m_sha.group(1) != sha:
        return None
    return float(m_tr.group(1))


# -------------------------------------------------------------- main legs

def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")
    return world, rank, local, dist


def reference_main(args, world, rank, dist):
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    vals, t0 = [], time.perf_counter()
    for s in range(args.warmup + args.steps):
        v, desc = oracle_sample(args.workload, 2, 1000 + s, min(cores, 2))
        if s >= args.warmup:
            vals.append(v)
    value = statistics.mean(vals)
    wall = time.perf_counter() - t0
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "resultants/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * wall / (args.steps + args.warmup),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int (Python big integers)",
            "data": "synthetic", "config": {"workload": WORKLOADS[args.workload]},
            "cpu_baseline": {"value": value, "unit": "resultants/s", "cores": min(cores, 2),
                             "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": "resultants/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def ours_main(args, world, rank, local, dist):
    import torch
    from paper_1010_1386_gb300 import rs

    torch.cuda.set_device(local)
    pairs = load_pairs(args.workload, args.pairs)
    npairs = len(pairs)
    ctx = rs.Context(device=local, timing=True)
    stream = torch.cuda.ExternalStream(ctx.stream, device=local)
    batch = ctx.batch(pairs)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=f"cuda:{local}")

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(local)

    for _ in range(args.warmup):
        batch.run()
        batch.sync()
    info = batch.info()

    # ---- timed region: batched, device-resident inputs
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    g1_ms, stage = [], {"images": [], "interp": [], "crt": []}
    barrier()
    with ClockSampler(local) as clocks:
        t_wall = time.perf_counter()
        for s in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
                ev[s][0].record(stream)
            batch.run()
            with torch.cuda.stream(stream):
                ev[s][1].record(stream)
            batch.sync()
            i = batch.info()
            stage["images"].append(i["ms_images"])
            stage["interp"].append(i["ms_interp"])
            stage["crt"].append(i["ms_crt"])
        barrier()
        t_wall = time.perf_counter() - t_wall
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = statistics.mean(step_ms)
    if dist is not None:
        t = torch.tensor([ms], device=f"cuda:{local}")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = world * npairs / (ms * 1e-3)

    # ---- per-instance form: same kernels, one pair per launch sequence
    per_inst = None
    if args.workload == "batch" and not args.no_per_instance:
        ctx1 = rs.Context(device=local, use_graphs=False, persistent=False)
        singles = [ctx1.batch([p]) for p in pairs]
        for b in singles:
            b.run()
        singles[-1].sync()
        s1 = torch.cuda.ExternalStream(ctx1.stream, device=local)
        pe = []
        for _ in range(max(1, min(args.steps, 3))):
            a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(s1):
                flush.zero_()
                a.record(s1)
            for b in singles:
                b.run()
            with torch.cuda.stream(s1):
                b_.record(s1)
            singles[-1].sync()
            pe.append(a.elapsed_time(b_))
        pms = statistics.mean(pe)
        per_inst = {"value": npairs / (pms * 1e-3), "unit": "resultants/s", "ms_per_step": pms,
                    "form": "one pair per launch sequence (G1 one block per tile, G2, G3), "
                            "no persistent kernel, no CUDA graph"}
        for b in singles:
            b.close()
        ctx1.close()

    # ---- end to end through the C ABI with host buffers
    e2e_ms = []
    for s in range(max(1, min(args.steps, 3))):
        barrier()
        t = time.perf_counter()
        batch.upload(pairs)
        batch.run()
        batch.results(raw=True)
        e2e_ms.append(1e3 * (time.perf_counter() - t))
    e2e_val = world * npairs / (statistics.mean(e2e_ms) * 1e-3)

    g1 = statistics.mean(stage["images"])
    algo_imad = 4.0 * (info["modmul_eval"] + info["modmul_prs"])
    clk = clocks.summary()
    sm_max = clk["sm_max_mhz"] or 2070.0
    peak = SM_COUNT * IMAD_PER_SM_CLK * sm_max * 1e6 / 1e12
    achieved = algo_imad / (g1 * 1e-3) / 1e12
    traffic = g1_traffic()

    line = {
        "metric": METRIC, "value": value, "unit": "resultants/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload] + ("" if npairs == 512 or args.workload != "batch"
                                                           else f" (first {npairs} pairs)"),
                   "pairs_per_gpu": npairs,
                   "images_per_step": info["images"],
                   "l2": "256 MiB written before every timed step (outside its events); "
                         "per-step working set (num/den images) %.0f MB" % (info["images"] * 8 / 1e6),
                   "parallelism": f"independent batches, {world} GPU(s)"},
        "images_per_s": world * info["images"] / (ms * 1e-3),
        "stage_ms": {k: statistics.mean(v) for k, v in stage.items()},
        "per_instance": per_inst,
        "batched_over_per_instance": (value / world / per_inst["value"]) if per_inst else None,
        "imad_frac_g1": achieved / peak,
        "roofline": {"bound": "alu", "kernel": "G1 (reduce + evaluate + univariate resultant)",
                     "achieved": achieved, "peak": peak, "unit": "TIMAD/s", "frac": achieved / peak,
                     "traffic": traffic,
                     "peak_source": f"derived: {SM_COUNT} SMs x {IMAD_PER_SM_CLK} IMAD/clk x "
                                    f"{sm_max:.0f} MHz (no integer peak in MEASURED_PEAKS.json)"},
        "clocks": clk,
        "e2e": {"value": e2e_val, "unit": "resultants/s",
                "h2d_bytes_per_step": info["input_bytes"], "d2h_bytes_per_step": info["output_bytes"]},
        "detections": {"unlucky_points": info["unlucky_points"],
                       "degenerate_images": info["degenerate_images"],
                       "unlucky_primes": info["unlucky_primes"]},
    }
    line["gpu_launches"] = args.steps * info["kernel_launches"]
    if rank == 0 and not args.no_baseline:
        cores = os.cpu_count() or 1
        v, desc = oracle_sample(args.workload, 8 if args.workload == "batch" else 2, 7,
                                min(cores, 8))
        line["cpu_baseline"] = {"value": v, "unit": "resultants/s", "cores": min(cores, 8),
                                "kind": "oracle", "sample": desc}
    if rank == 0:
        print(json.dumps(line), flush=True)
    batch.close()
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batch", choices=sorted(WORKLOADS))
    ap.add_argument("--no-baseline", action="store_true")
    ap.add_argument("--no-per-instance", action="store_true")
    ap.add_argument("--pairs", type=int, default=512,
                    help="profiling only: time the first PAIRS pairs of the batch")
    args = ap.parse_args()
    world, rank, local, dist = dist_setup(args)
    if args.impl == "reference":
        reference_main(args, world, rank, dist)
    else:
        ours_main(args, world, rank, local, dist)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
