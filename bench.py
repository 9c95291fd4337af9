"""Benchmark: exact bivariate resultants per second on one GB300 (or N, one
process per GPU, independent batches: weak scaling).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload batch|small|single|nongeneric|nongeneric-coprime|serving|shift|squarefree]
                    [--no-baseline] [--no-per-instance]

Prints ONE JSON line.  A step is one pass of the whole path (G1 reduce +
evaluate + univariate resultants, G2 interpolation, G3 CRT) over one batch of
synthetic input; the default workload is 512 pairs with per-pair deg_x,
deg_y ~ U[8, 40], bidegree-dense, coefficient bits in {16, 32, 64}.
``value`` is the batched throughput with inputs resident on the device;
``per_instance`` times the same kernels launched one pair at a time (no
persistence, no graphs); ``e2e`` goes through the C ABI with host buffers
(upload, run, result copy-back); ``cpu_baseline`` times the CPU oracle on a
bounded sample.  ``--workload serving`` runs a Poisson stream of 10,000
requests through the continuous-batching server and reports p50/p99 latency.
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
INTERP = {"auto": 0, "direct": 1, "transforms": 2, "triangular": 3, "tensor": 4}
SQF_METRIC = "square-free factorisations of Res_y(f, g) per second (R = c prod R_i^i), one GB300"
IMAD_PER_SM_CLK = 64  # nominal 32-bit integer multiply-add results per clock per SM
WORKLOADS = {
    "batch": "batched: 512 pairs in one run, per-pair deg_x, deg_y ~ U[8,40] shared by f and g, "
             "bidegree-dense, coefficient bits per pair in {16,32,64}, seed 2",
    "small": "single pair, dense total degree 6, coefficients uniform in [-2^10, 2^10], seed 0",
    "single": "single pair, dense total degree 30, signed 32-bit coefficients, seed 1",
    "nongeneric": "batch of 32: f = p q^2 (p, q dense total degrees 24 and 12, 64-bit coefficients), "
                  "g = df/dy (common factor q: Res_y = 0), seed 3",
    "nongeneric-coprime": "batch of 32: f = p q^2 as above, g = d(pq)/dy (coprime, Res_y with repeated "
                          "factors), seed 3",
    "serving": "Poisson stream of 10,000 requests, total degrees of f and g ~ U[8,64], coefficient bits "
               "~ U[16,128], total-degree-dense, seed 4",
    "squarefree": "square-free factorisation Res_y = c prod R_i^i of each pair of the non-generic "
                  "coprime batch (32 pairs, f = p q^2, g = d(pq)/dy, p and q dense total degrees 24 and "
                  "12, 64-bit coefficients, seed 3): one call through the C ABI per step, host buffers "
                  "in and out",
    "shift": "both projections Res_y and Res_x of all 10 pairs of five random curves (total degree "
             "--shift-deg, dense or --shift-sparse, 16-bit coefficients) multiplied by 2^k "
             "(--shift-k) with the constant term raised by one, seed 5: 20 resultants",
}


SHIFT = (15, 512, False)  # shift workload (degree, k, sparse); main() sets it from the flags


def load_pairs(workload, npairs=None, rank=0, args=None):
    """The workload's pairs; under weak scaling rank r > 0 draws its own
    batch of the same distribution (seed + 1000 r).  Uses the seeded
    generators only (no library)."""
    from paper_1010_1386_gb300 import inputs
    from paper_1010_1386_gb300.sharding import rank_seed
    if workload == "shift":
        deg, k, sparse = (args.shift_deg, args.shift_k, args.shift_sparse) if args else SHIFT
        base = inputs.workload_shift(rank_seed(5, rank), deg, sparse, k)
        pairs = base + [(inputs.swap_xy(f), inputs.swap_xy(g)) for f, g in base]  # R^{(y)}, then R^{(x)}
        return pairs[:npairs] if npairs else pairs
    if workload == "batch":
        pairs = inputs.workload_batch(rank_seed(2, rank), n=512)
    elif workload == "small":
        pairs = inputs.workload_small(0)
    elif workload == "single":
        pairs = inputs.workload_single(1)
    elif workload == "nongeneric":
        pairs = inputs.workload_nongeneric(rank_seed(3, rank), n=32)
    elif workload == "nongeneric-coprime":
        pairs = inputs.workload_nongeneric(rank_seed(3, rank), n=32, coprime=True)
    else:
        pairs = inputs.workload_serving(4, n=npairs or 10000)[0]
    return pairs[:npairs] if npairs else pairs


# ------------------------------------------------------------ CPU oracle leg

def cpu_threads():
    return os.cpu_count() or 1


def oracle_sample(workload, seconds, seed, threads, args=None):
    """Time the independent modular oracle O2 (``oracle.modular``: its own
    plan, every image, interpolation and CRT -- the whole algorithm) on a
    seeded random sample of the workload's pairs, on ``threads`` host
    threads.  Chunks of ``threads`` pairs are drawn without replacement and
    run until ``seconds`` of wall time are spent (the whole workload if it
    is done first; a one-pair workload is repeated).  Returns
    (resultants/s, pairs timed, description)."""
    import random
    from oracle import modular
    modular.load()
    pairs = load_pairs(workload, 512 if workload == "serving" else None, 0, args)
    order = list(range(len(pairs)))
    random.Random(seed).shuffle(order)
    done, wall, pos = 0, 0.0, 0
    while wall < seconds:
        if pos >= len(order):
            if len(pairs) > 1:
                break
            pos = 0
        chunk = order[pos:pos + threads]
        pos += len(chunk)
        t = time.perf_counter()
        modular.resultants([pairs[i] for i in chunk], threads=threads)
        wall += time.perf_counter() - t
        done += len(chunk)
    total = len(pairs) if workload != "serving" else 10000
    desc = (f"measured: oracle O2 (C, whole algorithm: plan, Euclid/Sylvester images at x = 0..D, "
            f"Lagrange interpolation, CRT) on {done} {'random ' if len(pairs) > 1 else ''}pair(s) "
            f"of the {total} in {wall:.1f} s wall, {threads} threads")
    return done / wall, done, desc


def _oracle_sqf(args):
    f, g = args
    from oracle import exact, squarefree
    t = time.perf_counter()
    squarefree.squarefree(exact.resultant_y(f, g))
    return time.perf_counter() - t


def oracle_sqf_sample(npairs, seed, cores):
    """Time the oracle (exact resultant, then Yun over Z) on ``npairs`` pairs
    of the non-generic coprime generator at reduced degrees (p, q of total
    degrees 4 and 2; at 6 and 3 one pair already takes the oracle two
    minutes, the full-size pairs far longer).  Returns
    (factorisations/s over ``cores`` processes, description)."""
    from paper_1010_1386_gb300 import inputs
    pairs = inputs.workload_nongeneric(seed, n=npairs, deg_p=4, deg_q=2, bits=64, coprime=True)
    jobs = [(f.to_ints(), g.to_ints()) for f, g in pairs]
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(cores, len(jobs))) as pool:
        times = pool.map(_oracle_sqf, jobs)
    value = cores / statistics.mean(times)
    desc = (f"oracle exact Res_y then Yun over Z for {len(jobs)} pairs of the same generator at "
            f"reduced size (p, q total degrees 4 and 2; mean {statistics.mean(times):.2f} s each); "
            f"{cores} processes")
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

def _traffic_paths():
    return (os.path.join(ROOT, "profiles", "g1_traffic.json"),
            os.path.join(ROOT, "paper_1010_1386_gb300", "csrc", "kernels_g1.cu"))


def _sha256(path):
    return hashlib.sha256(open(path, "rb").read()).hexdigest()


def g1_traffic():
    """DRAM bytes of one G1 stage of the default workload from the record
    that ``--record-traffic`` wrote from an ncu capture, if that capture was
    taken on the current G1 source; else None."""
    path, src = _traffic_paths()
    try:
        rec = json.load(open(path))
        if rec["kernels_g1_sha256"] != _sha256(src):
            return None
        return float(rec["dram_bytes_per_stage"])
    except (OSError, KeyError, ValueError):
        return None


def record_traffic(csv_path, command):
    """Write profiles/g1_traffic.json from an ncu --csv log of the G1 launches
    (metrics dram__bytes_read.sum and dram__bytes_write.sum, one value per
    launch): the DRAM bytes of the last complete step, i.e. the last launch
    of each G1 kernel instance name."""
    import csv
    rows = [r for r in csv.reader(open(csv_path)) if r]
    hdr = next(i for i, r in enumerate(rows) if "Metric Name" in r)
    h = rows[hdr]
    ki, mi, vi, ui = h.index("Kernel Name"), h.index("Metric Name"), h.index("Metric Value"), h.index("Metric Unit")
    idi = h.index("ID")
    scale = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}
    per = {}
    for r in rows[hdr + 1:]:
        if "g1_kernel" not in r[ki] or not r[mi].startswith("dram__bytes_"):
            continue
        per.setdefault(r[ki], {}).setdefault(int(r[idi]), 0.0)
        per[r[ki]][int(r[idi])] += float(r[vi].replace(",", "")) * scale.get(r[ui], 1)
    last = {k: v[max(v)] for k, v in per.items()}
    path, src = _traffic_paths()
    rec = {"kernel": "G1 (all register-capacity launches of one step)",
           "dram_bytes_per_stage": sum(last.values()), "per_launch": last,
           "kernels_g1_sha256": _sha256(src), "command": command,
           "note": "dram__bytes_read.sum + dram__bytes_write.sum of the last launch of each G1 kernel"}
    with open(path, "w") as fh:
        json.dump(rec, fh, indent=1, sort_keys=True)
        fh.write("\n")
    print(json.dumps(rec))


# -------------------------------------------------------------- helpers

def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")
    return world, rank, local, dist


def barrier(dist, local):
    import torch
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize(local)


def max_over_ranks(dist, local, value):
    from paper_1010_1386_gb300.sharding import max_over_ranks as mor
    return mor(value, dist, device=f"cuda:{local}")


_PEAK = {}


def int_peak():
    """The device's integer multiply-add throughputs, measured once per
    process by the library's probe (rs_measure_int_peak) before any timed
    region."""
    if not _PEAK:
        from paper_1010_1386_gb300 import rs
        _PEAK.update(rs.measure_int_peak())
    return _PEAK


def roofline(info, g1_ms, clk, kernel="G1 (reduce + evaluate + univariate resultant)"):
    """G1's algorithmic IMAD rate (4 multiply-adds per modular product of
    the evaluation and the remainder sequence) against the measured
    mad.lo.u32 peak of this device."""
    pk = int_peak()
    peak = pk["mad_lo_u32"] / 1e12
    achieved = 4.0 * (info["modmul_eval"] + info["modmul_prs"]) / (g1_ms * 1e-3) / 1e12
    sm_max = clk["sm_max_mhz"] or pk["clock_max_mhz"]
    derived = pk["sms"] * IMAD_PER_SM_CLK * sm_max * 1e6 / 1e12
    return {"bound": "alu", "kernel": kernel,
            "achieved": achieved, "peak": peak, "unit": "TIMAD/s", "frac": achieved / peak,
            "traffic": None,
            "peak_source": "measured: rs_measure_int_peak, independent mad.lo.u32 chains on all %d SMs "
                           "(%.1f per clock per SM at the %.0f MHz maximum clock)"
                           % (pk["sms"], pk["mad_lo_u32"] / (pk["sms"] * pk["clock_max_mhz"] * 1e6),
                              pk["clock_max_mhz"]),
            "probe": {"mad_lo_u32_T": pk["mad_lo_u32"] / 1e12, "mad_wide_u32_T": pk["mad_wide_u32"] / 1e12,
                      "mad_hi_u32_T": pk["mad_hi_u32"] / 1e12, "mad_wide_s32_T": pk["mad_wide_s32"] / 1e12,
                      "montgomery_step_T": pk["mont_update"] / 1e12, "sms": pk["sms"]},
            "derived_peak": derived, "frac_of_derived": achieved / derived}


def whole_path_work(info, npairs, ms, peak):
    """Algorithmic modular products of one step by stage (a3 evaluation, a4
    univariate resultants, a5 interpolation counted in its direct
    convolution form, a6 Garner digits) and the whole path's rate at 4 IMAD
    per product against the same derived peak as the G1 roofline."""
    parts = {"eval": info["modmul_eval"], "prs": info["modmul_prs"], "interp": info["modmul_interp"],
             "crt": info["modmul_crt"]}
    total = sum(parts.values())
    rate = 4.0 * total / (ms * 1e-3) / 1e12
    return {"unit": "modular products per step (interp: direct-convolution count)", **parts,
            "total": total, "per_resultant": total / max(npairs, 1),
            "whole_path_timad_s": rate, "whole_path_frac": rate / peak}


def base_line(args, world, value, ms, workload_desc, extra_cfg):
    return {"metric": METRIC, "value": value, "unit": "resultants/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": dict({"workload": workload_desc,
                            "parallelism": f"independent batches, {world} GPU(s); rank r > 0 "
                                           "draws its own batch (seed + 1000 r)"}, **extra_cfg)}


def add_cpu_baseline(line, args, rank):
    """``cpu_baseline``: the oracle as it stands, timed on this host's cores
    (rank 0 at N = 1 only; about args.baseline_seconds of CPU work)."""
    if rank != 0 or args.no_baseline or int(os.environ.get("WORLD_SIZE", "1")) > 1:
        return
    threads = cpu_threads()
    if args.workload == "squarefree":
        v, desc = oracle_sqf_sample(threads, 7, threads)
        line["cpu_baseline"] = {"value": v, "unit": "factorisations/s", "cores": threads, "kind": "oracle",
                                "sample": desc}
        return
    v, n, desc = oracle_sample(args.workload, args.baseline_seconds, 7, threads, args)
    line["cpu_baseline"] = {"value": v, "unit": "resultants/s", "cores": threads, "kind": "oracle",
                            "sample": desc, "pairs": n}


# ------------------------------------------------------------------ legs

def reference_main(args, world, rank, dist):
    """The reference arm: the oracle O2 on this host's cores, the same
    workload, metric and unit as the GPU arm.  Each step is a seeded random
    sample of the workload (``threads`` pairs, or the whole workload if it
    is smaller; a one-pair workload runs once per step); value = pairs timed
    / wall time of the timed steps.  Loads no GPU library.  Under torchrun
    only rank 0 works."""
    if rank != 0:
        return
    import random
    from oracle import modular
    threads = cpu_threads()
    sqf = args.workload == "squarefree"
    unit = "factorisations/s" if sqf else "resultants/s"
    if sqf:
        vals = []
        desc = ""
        t0 = time.perf_counter()
        for s in range(args.warmup + args.steps):
            v, desc = oracle_sqf_sample(threads, 1000 + s, threads)
            if s >= args.warmup:
                vals.append(v)
        value = statistics.mean(vals)
        ms = 1000.0 * (time.perf_counter() - t0) / (args.steps + args.warmup)
    else:
        modular.load()
        pairs = load_pairs(args.workload, 512 if args.workload == "serving" else None, 0, args)
        per_step = min(len(pairs), threads)
        done, wall = 0, 0.0
        for s in range(args.warmup + args.steps):
            idx = random.Random(1000 + s).sample(range(len(pairs)), per_step)
            t = time.perf_counter()
            modular.resultants([pairs[i] for i in idx], threads=threads)
            dt = time.perf_counter() - t
            if s >= args.warmup:
                done += per_step
                wall += dt
        value = done / wall
        ms = 1000.0 * wall / args.steps
        desc = (f"measured: oracle O2 (C, whole algorithm: plan, Euclid/Sylvester images at x = 0..D, "
                f"Lagrange interpolation, CRT), {args.steps} timed steps of {per_step} seeded random "
                f"pair(s) each ({done} pairs, {wall:.1f} s wall), {threads} threads")
    line = base_line(args, 1, value, ms, WORKLOADS[args.workload], {})
    if sqf:
        line.update({"metric": SQF_METRIC, "unit": unit})
    line.update({"impl": "reference", "dtype": "u32 modular (64-bit products), bignum CRT",
                 "cpu_baseline": {"value": value, "unit": unit, "cores": threads,
                                  "kind": "oracle", "sample": desc},
                 "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0,
                         "d2h_bytes_per_step": 0}})
    print(json.dumps(line), flush=True)


def batch_main(args, world, rank, local, dist):
    import torch
    from paper_1010_1386_gb300 import rs

    torch.cuda.set_device(local)
    pairs = load_pairs(args.workload, args.pairs, rank, args)
    npairs = len(pairs)
    ctx = rs.Context(device=local, timing=True, autotune_cache=args.autotune_cache,
                     univariate=args.univariate, g2_form=INTERP[args.interp])
    int_peak()  # the integer-pipe probe runs before anything is timed
    stream = torch.cuda.ExternalStream(ctx.stream, device=local)
    t_tune = time.perf_counter()
    batch = ctx.batch(pairs)  # tunes the G1 launch of every class of the batch first
    t_tune = time.perf_counter() - t_tune
    tuned = rs.autotune_entries()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=f"cuda:{local}")
    for _ in range(args.warmup):
        batch.run()
        batch.sync()
    info = batch.info()

    # timed region: device-resident inputs
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    stage = {"images": [], "interp": [], "crt": []}
    barrier(dist, local)
    with ClockSampler(local) as clocks:
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
        barrier(dist, local)
    ms = max_over_ranks(dist, local, statistics.mean(a.elapsed_time(b) for a, b in ev))
    value = world * npairs / (ms * 1e-3)

    per_inst = None
    if npairs > 1 and not args.no_per_instance:
        ctx1 = rs.Context(device=local, use_graphs=False, persistent=False, univariate=args.univariate,
                          g2_form=INTERP[args.interp])
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

    # End to end through the C ABI with host buffers: every step uploads its
    # inputs, runs, and copies its results back and trims them.  Sequential:
    # one prepared batch, step after step.  Pipelined: three prepared batches
    # on three streams rotate; a step's results are taken just before its
    # batch is reused, so its result copy and trim (and the next uploads)
    # overlap the runs queued behind it (the same transfers, overlapped).
    e2e_steps = max(8, min(2 * args.steps, 16))
    e2e_ms = []
    batch.upload(pairs)  # one untimed end-to-end pass (host buffers, staging pages)
    batch.run()
    batch.results(raw=True)
    for _ in range(max(3, min(args.steps, 5))):
        barrier(dist, local)
        t = time.perf_counter()
        batch.upload(pairs)
        batch.run()
        batch.results(raw=True)
        e2e_ms.append(1e3 * (time.perf_counter() - t))
    e2e_seq = world * npairs / (max_over_ranks(dist, local, statistics.mean(e2e_ms)) * 1e-3)
    depth = 3
    streams = [torch.cuda.Stream(device=local) for _ in range(depth)]
    pipe = [ctx.batch(pairs, stream=st.cuda_stream) for st in streams]
    for b in pipe:  # untimed: staging pages, graph capture
        b.upload(pairs)
        b.run()
        b.results(raw=True)
    # Two orchestrations of the same calls, both timed: "chained", where each
    # run waits for the previous run's kernels (an event on the previous
    # stream), so uploads, result copies and trims overlap the running step
    # but the steps' kernels do not interleave (on a batch that fills the GPU,
    # three batches' kernels sharing the SMs took 1 to 3 ms a step more);
    # and "free", where consecutive steps may overlap on the device (better
    # when one step leaves the GPU mostly idle: a single pair, few resultants
    # with many primes).  GPU span: from the first upload to the end of the
    # last run.
    def pipelined(chained):
        barrier(dist, local)
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local) as clk_e2e:  # the pipelined loop keeps the GPU busy for longer
            t = time.perf_counter()
            prev_run = None
            for s in range(e2e_steps):
                b, st = pipe[s % depth], streams[s % depth]
                if s >= depth:
                    b.results(raw=True)  # step s - depth: its results before the batch is reused
                if s == 0:
                    g0.record(streams[0])
                b.upload(pairs)
                if chained and prev_run is not None:
                    st.wait_event(prev_run)
                b.run()
                prev_run = torch.cuda.Event()
                prev_run.record(st)
                if s == e2e_steps - 1:
                    g1.record(st)
            for s in range(max(0, e2e_steps - depth), e2e_steps):
                pipe[s % depth].results(raw=True)
            ms_ = 1e3 * (time.perf_counter() - t) / e2e_steps
        torch.cuda.synchronize(local)
        ms_ = max_over_ranks(dist, local, ms_)
        return {"value": world * npairs / (ms_ * 1e-3), "ms_per_step": ms_,
                "gpu_ms_per_step": g0.elapsed_time(g1) / e2e_steps, "clocks": clk_e2e.summary()}

    forms = {"chained": pipelined(True), "free": pipelined(False)}
    best = max(forms, key=lambda k: forms[k]["value"])
    pipe_ms, pipe_gpu_ms, clocks_e2e_summary = (forms[best]["ms_per_step"], forms[best]["gpu_ms_per_step"],
                                                forms[best]["clocks"])
    e2e_val = forms[best]["value"]
    for b in pipe:
        b.close()

    clk = clocks.summary()
    g1 = statistics.mean(stage["images"])
    if args.univariate == "schur":
        rf = roofline(info, g1, clk, "G1, Schur variant (reduce + evaluate + Schur on generators + "
                                     "elimination fallback)")
    else:
        rf = roofline(info, g1, clk)
    if args.workload == "batch" and npairs == 512 and args.univariate == "prs":
        rf["traffic"] = g1_traffic()
    desc = WORKLOADS[args.workload] + ("" if args.pairs is None else f" (first {npairs} pairs)")
    line = base_line(args, world, value, ms, desc,
                     {"pairs_per_gpu": npairs, "images_per_step": info["images"],
                      "univariate": ("Schur algorithm on displacement generators, one warp per image"
                                     if args.univariate == "schur" else
                                     "division-free remainder sequence, one thread per image"),
                      "interpolation": {"auto": "convolutions per length group: direct, transforms or all pairs of "
                                                "a prime as one exact tensor-core product (bf16 digits, fp32 "
                                                "accumulation), as the tuner chose",
                                        "direct": "direct convolutions", "transforms": "transforms",
                                        "triangular": "triangular factorisation of the Vandermonde "
                                                      "system (Bjorck-Pereyra stages)",
                                        "tensor": "convolutions of all pairs of a prime as exact matrix "
                                                  "products on the tensor cores (bf16 digits, fp32 "
                                                  "accumulation)"}[args.interp],
                      "l2": "256 MiB written before every timed step (outside its events); per-step "
                            "working set (num/den images) %.0f MB" % (info["images"] * 8 / 1e6)})
    line.update({
        "images_per_s": world * info["images"] / (ms * 1e-3),
        "stage_ms": {k: statistics.mean(v) for k, v in stage.items()},
        "per_instance": per_inst,
        "batched_over_per_instance": (value / world / per_inst["value"]) if per_inst else None,
        "imad_frac_g1": rf["frac"],
        "roofline": rf,
        "work": whole_path_work(info, npairs, ms, rf["peak"]),
        "gpu_launches": args.steps * info["kernel_launches"],
        "clocks": clk,
        "e2e": {"value": e2e_val, "unit": "resultants/s", "h2d_bytes_per_step": info["input_bytes"],
                "d2h_bytes_per_step": info["output_bytes"],
                "form": "pipelined: three prepared batches on three streams rotate (a step's result "
                        "copy and trim just before its batch is reused), %d steps; the better of two "
                        "orchestrations: %s (chained: each run starts after the previous run's "
                        "kernels; free: runs may overlap)" % (e2e_steps, best),
                "clocks": clocks_e2e_summary,
                "gpu_ms_per_step": pipe_gpu_ms,
                "orchestrations": {k: {"value": v["value"], "gpu_ms_per_step": v["gpu_ms_per_step"]}
                                   for k, v in forms.items()},
                "sequential": {"value": e2e_seq, "unit": "resultants/s",
                               "form": "one prepared batch: upload, run, results, step after step"}},
        "autotune": {"build_s": t_tune,
                     "classes": [{"stage": "G1" if e["kind"] == 0 else "G2", "cap": e["cap"],
                                  "lg_points": e["lg_points"], "lg_images": e["lg_images"],
                                  "choice": (e["choice"] if e["kind"] == 0 else
                                             ["direct", "transforms", "tensor cores"][e["choice"]]),
                                  "persistent": e["persistent"],
                                  "gain": (e["ms_default"] / e["ms_best"]) if e["ms_best"] else None}
                                 for e in tuned]},
        "detections": {"unlucky_points": info["unlucky_points"],
                       "degenerate_images": info["degenerate_images"],
                       "unlucky_primes": info["unlucky_primes"]},
    })
    if args.workload == "batch" and not args.no_other_configs and world == 1 and args.pairs is None:
        line["configs"] = other_configs(ctx, local, args.steps, flush, stream)
    add_cpu_baseline(line, args, rank)
    if rank == 0:
        print(json.dumps(line), flush=True)
    batch.close()
    ctx.close()


def squarefree_main(args, world, rank, local, dist):
    """One rs_squarefree_batch call per step (GPU pass over the factors'
    primes, Yun mod p, CRT of the factors, primitive parts on the host); the
    resultant alone on the same pairs is timed beside it."""
    import torch
    from paper_1010_1386_gb300 import rs

    torch.cuda.set_device(local)
    pairs = load_pairs("nongeneric-coprime", args.pairs, rank, args)
    npairs = len(pairs)
    ctx = rs.Context(device=local, timing=True, autotune_cache=args.autotune_cache)
    batch = ctx.batch(pairs)
    for _ in range(args.warmup):
        batch.run()
        batch.sync()
    res_ms = []
    for _ in range(max(3, min(args.steps, 5))):
        batch.run()
        batch.sync()
        res_ms.append(batch.info()["ms_total"])
    batch.close()
    maxm = 4
    for _ in range(args.warmup):
        st = ctx.squarefree_batch(pairs, maxm, raw=True)
        assert all(c == 0 for c in st), st
    times, infos = [], []
    barrier(dist, local)
    with ClockSampler(local) as clocks:
        for _ in range(args.steps):
            t = time.perf_counter()
            st = ctx.squarefree_batch(pairs, maxm, raw=True)
            times.append(1e3 * (time.perf_counter() - t))
            infos.append(ctx.squarefree_info())
        barrier(dist, local)
    assert all(c == 0 for c in st), st
    ms = max_over_ranks(dist, local, statistics.mean(times))
    value = world * npairs / (ms * 1e-3)
    last = infos[-1]
    bi = last["batch"]
    mean = lambda k: statistics.mean(i[k] for i in infos)
    bmean = lambda k: statistics.mean(i["batch"][k] for i in infos)
    clk = clocks.summary()
    rf = roofline(bi, bmean("ms_images"), clk)
    out = ctx.squarefree_batch(pairs[:1], maxm)[0]
    line = base_line(args, world, value, ms, WORKLOADS["squarefree"],
                     {"pairs_per_gpu": npairs, "max_mult": maxm, "images_per_step": bi["images"],
                      "primes_per_pair": bi["primes_total"] / max(1, bi["pairs"]),
                      "l2": "inputs and the per-step working set (%.0f MB of images) exceed L2"
                            % (bi["images"] * 8 / 1e6)})
    line.update({
        "metric": SQF_METRIC, "unit": "factorisations/s",
        "stage_ms": {"G1": bmean("ms_images"), "G2": bmean("ms_interp"), "yun": bmean("ms_yun"),
                     "G3 (R)": bmean("ms_crt"), "lift (factor CRT)": mean("ms_lift"),
                     "host (selection, contents, primitive parts)": mean("ms_host"),
                     "host: primitive parts": mean("ms_primitive"),
                     "host: analyse": mean("ms_analyse"),
                     "host: R's contents": mean("ms_contents"),
                     "host: lifted limbs fetch": mean("ms_fetch"),
                     "call": mean("ms_total")},
        "resultant_only": {"ms_per_step": statistics.mean(res_ms),
                           "value": npairs / (statistics.mean(res_ms) * 1e-3), "unit": "resultants/s",
                           "note": "same pairs, device-resident inputs, resultant primes only"},
        "factor_degrees_pair0": [(m, len(r) - 1) for m, r in out[1]],
        "primitive_parts_on_device": "%d of %d factors" % (last["factors_device"], last["factors"]),
        "roofline": rf,
        "gpu_launches": args.steps * (bi["kernel_launches"] + 3),
        "clocks": clk,
        "e2e": {"value": value, "unit": "factorisations/s",
                "h2d_bytes_per_step": last["h2d_bytes"], "d2h_bytes_per_step": last["d2h_bytes"],
                "note": "the call is end to end (host inputs, host outputs); value is the same number; "
                        "bytes are the call's own copies (inputs and CRT descriptors in; R's limbs, "
                        "Yun headers and lifted factors out)"},
    })
    add_cpu_baseline(line, args, rank)
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()


def measure_serving(local, n, load, inflight, max_batch, dist=None, clocks=None):
    """Closed-loop saturation pass, then a Poisson stream at ``load`` x that
    throughput through the continuous-batching server; every request crosses
    the C ABI with host buffers.  Returns the measurements as a dict."""
    import numpy as np
    from paper_1010_1386_gb300 import inputs, rs

    pairs, gaps = inputs.workload_serving(4, n=n)
    ctx = rs.Context(device=local)
    for k in (16, 64, 256):  # the server never tunes: warm the tuner cache with batches of a mix
        ctx.autotune(pairs[:k])
    srv = rs.Server(ctx, max_inflight=inflight, max_batch=max_batch)
    for f, g in pairs[: min(n, 256)]:  # warm-up: tables, streams, pinned staging
        srv.wait(srv.submit(f, g))

    def run_stream(times):
        """Submit pair i at times[i] (seconds from start; None = at once)."""
        tickets = [None] * n

        def producer():
            t0 = time.perf_counter()
            for i, (f, g) in enumerate(pairs):
                if times is not None:
                    dt = times[i] - (time.perf_counter() - t0)
                    if dt > 0:
                        time.sleep(dt)
                tickets[i] = srv.submit(f, g)
        t_start = time.perf_counter()
        th = threading.Thread(target=producer)
        th.start()
        lat, out_bytes = [], 0
        for i in range(n):
            while tickets[i] is None:
                time.sleep(0.0001)
            (deg, limbs, _), ms = srv.wait(tickets[i], raw=True)  # limbs into a host buffer, no Python ints
            lat.append(ms)
            out_bytes += 4 * max(deg + 1, 0) * limbs
        th.join()
        return time.perf_counter() - t_start, lat, out_bytes

    barrier(dist, local)
    sat_s, sat_lat, _ = run_stream(None)
    sat = n / sat_s
    rate = load * sat
    arrivals = np.cumsum(gaps) / rate
    wall, lat, out_bytes = run_stream(arrivals)
    barrier(dist, local)
    st = srv.stats()
    srv.stop()
    ctx.close()
    lat_sorted = sorted(lat)
    return {"requests": n, "wall_s": wall, "value": n / wall, "unit": "resultants/s",
            "arrival_rate_per_s": rate, "load_vs_saturation": load,
            "latency_ms": {"p50": lat_sorted[len(lat) // 2],
                           "p99": lat_sorted[min(len(lat) - 1, int(0.99 * len(lat)))],
                           "mean": statistics.mean(lat)},
            "saturation": {"value": sat, "unit": "resultants/s", "p50_ms": sorted(sat_lat)[n // 2]},
            "server": {k: st[k] for k in ("batches", "peak_inflight_batches", "peak_running", "failed")},
            "kernel_launches": st["kernel_launches"],
            "h2d_bytes": int(sum(f.coeffs.nbytes + g.coeffs.nbytes for f, g in pairs)),
            "d2h_bytes": out_bytes, "max_inflight_batches": inflight, "max_batch": max_batch}


def serving_main(args, world, rank, local, dist):
    """Closed-loop saturation pass, then a Poisson stream at --load x that
    throughput through the continuous-batching server."""
    import torch

    torch.cuda.set_device(local)
    with ClockSampler(local) as clocks:
        r = measure_serving(local, args.pairs or 10000, args.load, args.inflight, args.max_batch, dist)
    wall = max_over_ranks(dist, local, r["wall_s"])
    n = r["requests"]
    value = world * n / wall
    line = base_line(args, world, value, 1e3 * wall, WORKLOADS["serving"],
                     {"requests": n, "arrival_rate_per_s": r["arrival_rate_per_s"],
                      "load_vs_saturation": args.load, "max_inflight_batches": args.inflight,
                      "max_batch": args.max_batch})
    line.update({
        "steps": 1,
        "latency_ms": r["latency_ms"],
        "saturation": r["saturation"],
        "server": r["server"],
        "gpu_launches": r["kernel_launches"],
        "clocks": clocks.summary(),
        "e2e": {"value": value, "unit": "resultants/s", "h2d_bytes_per_step": r["h2d_bytes"],
                "d2h_bytes_per_step": r["d2h_bytes"],
                "note": "every request crosses the C ABI with host buffers; latency is submit to result; "
                        "the step is the whole stream, d2h the result limbs handed back"},
    })
    add_cpu_baseline(line, args, rank)
    if rank == 0:
        print(json.dumps(line), flush=True)


def measure_batch(ctx, pairs, steps, warmup, stream, flush, e2e_steps=0):
    """Device-timed steps of one prepared batch (inputs resident, L2 flushed
    before each step outside its events), then ``e2e_steps`` end-to-end
    steps through the C ABI with host buffers (upload, run, results)."""
    import torch
    b = ctx.batch(pairs)
    for _ in range(warmup):
        b.run()
        b.sync()
    ms, stage = [], {"images": [], "interp": [], "crt": []}
    for _ in range(steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            flush.zero_()
            e0.record(stream)
        b.run()
        with torch.cuda.stream(stream):
            e1.record(stream)
        b.sync()
        ms.append(e0.elapsed_time(e1))
        i = b.info()
        for k, key in (("images", "ms_images"), ("interp", "ms_interp"), ("crt", "ms_crt")):
            stage[k].append(i[key])
    info = b.info()
    out = {"value": len(pairs) / (statistics.mean(ms) * 1e-3), "unit": "resultants/s",
           "ms_per_step": statistics.mean(ms), "stage_ms": {k: statistics.mean(v) for k, v in stage.items()},
           "images_per_step": info["images"], "steps": steps, "gpu_launches": steps * info["kernel_launches"]}
    if e2e_steps:
        b.upload(pairs)
        b.run()
        b.results(raw=True)
        t = time.perf_counter()
        for _ in range(e2e_steps):
            b.upload(pairs)
            b.run()
            b.results(raw=True)
        e2e_ms = 1e3 * (time.perf_counter() - t) / e2e_steps
        out["e2e"] = {"value": len(pairs) / (e2e_ms * 1e-3), "unit": "resultants/s",
                      "h2d_bytes_per_step": info["input_bytes"], "d2h_bytes_per_step": info["output_bytes"],
                      "form": "one prepared batch: upload, run, results, step after step"}
    b.close()
    return out


def other_configs(ctx, local, steps, flush, stream):
    """Compact records of the other configurations, on the same GPU right
    after the headline workload: the single dense degree-30 pair (with its
    end-to-end rate), the coprime non-generic batch of 32 (g = (pq)_y, the
    non-zero variant of f = p q^2, g = f_y), both projections of the dense
    degree-15 shift workload at k = 2048 (about 2,000 primes per resultant;
    with its end-to-end rate) and the serving stream (10,000 requests
    at 0.8 of the measured saturation rate)."""
    from paper_1010_1386_gb300 import inputs
    out = {}
    out["c1_single_dense30"] = measure_batch(ctx, inputs.workload_single(1), max(steps, 10), 3, stream, flush,
                                             e2e_steps=20)
    out["c3p_nongeneric_coprime_32"] = measure_batch(ctx, inputs.workload_nongeneric(3, n=32, coprime=True),
                                                     max(3, min(steps, 5)), 2, stream, flush)
    base = inputs.workload_shift(5, 15, False, 2048)
    shift = base + [(inputs.swap_xy(f), inputs.swap_xy(g)) for f, g in base]
    out["shift_dense15_k2048"] = measure_batch(ctx, shift, max(3, min(steps, 10)), 3, stream, flush, e2e_steps=10)
    srv = measure_serving(local, 10000, 0.8, 3, 256)
    out["c4_serving_10000"] = {k: srv[k] for k in ("value", "unit", "latency_ms", "saturation",
                                                   "arrival_rate_per_s", "load_vs_saturation", "wall_s")}
    out["c4_serving_10000"]["form"] = ("Poisson arrivals at 0.8 of the closed-loop saturation rate, every "
                                       "request through the C ABI with host buffers (value is end to end)")
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batch", choices=sorted(WORKLOADS))
    ap.add_argument("--no-baseline", action="store_true")
    ap.add_argument("--no-per-instance", action="store_true")
    ap.add_argument("--no-other-configs", action="store_true",
                    help="batch workload: skip the compact records of the single degree-30 pair, "
                         "the coprime non-generic batch, the k = 2048 shift workload and the "
                         "serving stream")
    ap.add_argument("--record-traffic", default=None, metavar="CSV",
                    help="write profiles/g1_traffic.json from an ncu --csv log of the G1 launches and exit")
    ap.add_argument("--record-command", default="", help="the ncu command that wrote CSV (stored with it)")
    ap.add_argument("--baseline-seconds", type=float, default=15.0,
                    help="wall seconds of oracle work for cpu_baseline")
    ap.add_argument("--shift-deg", type=int, default=15, help="shift workload: total degree (9 or 15)")
    ap.add_argument("--shift-k", type=int, default=512, help="shift workload: coefficients times 2^k")
    ap.add_argument("--shift-sparse", action="store_true", help="shift workload: sparse curves")
    ap.add_argument("--univariate", default="prs", choices=["prs", "schur"],
                    help="univariate resultants mod p: remainder sequence (default) or the Schur "
                         "algorithm on displacement generators (comparison variant)")
    ap.add_argument("--interp", default="auto", choices=sorted(INTERP),
                    help="interpolation form: convolutions chosen per pair (auto), direct, transforms, "
                         "or the triangular factorisation of the Vandermonde system (comparison)")
    ap.add_argument("--autotune-cache", default=None,
                    help="tuner cache file read before and written after the run")
    ap.add_argument("--pairs", type=int, default=None,
                    help="time only the first PAIRS pairs / requests (profiling)")
    ap.add_argument("--load", type=float, default=0.8, help="serving: arrival rate / saturation")
    ap.add_argument("--inflight", type=int, default=3, help="serving: concurrent micro-batches")
    ap.add_argument("--max-batch", type=int, default=256, help="serving: requests per micro-batch")
    args = ap.parse_args()
    if args.record_traffic:
        record_traffic(args.record_traffic, args.record_command)
        return
    global SHIFT
    SHIFT = (args.shift_deg, args.shift_k, args.shift_sparse)
    world, rank, local, dist = dist_setup(args)
    if args.impl == "reference":
        reference_main(args, world, rank, dist)
    elif args.workload == "serving":
        serving_main(args, world, rank, local, dist)
    elif args.workload == "squarefree":
        squarefree_main(args, world, rank, local, dist)
    else:
        batch_main(args, world, rank, local, dist)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
